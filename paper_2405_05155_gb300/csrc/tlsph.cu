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
#include <algorithm>

#include "common.cuh"
#include "tiles.cuh"
#include "async.cuh"

namespace {

template <typename R>
struct TLK {
    R coef, inv_h;       // Wendland gs coefficient and 1/h
    R inv_rho0, dt, lam, G;
    int law;
    R half[3], Lh[3], Ll[3];
    R S[3], Sl[3];       // float32 path: cell size (hi + lo) of the cell-relative positions
    int ncell[3];
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
// Each neighbour record is a 32-byte line read with one 256-bit load:
//   RD [n][8]   3D (ox, oy, oz, cell, vx, vy, vz, V0)   2D (ox, oy, cell, V0, vx, vy, 0, 0)
//   RM [n][16]  3D (ox, oy, oz, cell, M00, M10, M20, V0, M01, M11, M21, 0, M02, M12, M22, 0)
//   RM [n][8]   2D (ox, oy, cell, V0, M00, M10, M01, M11)
// Positions are cell-relative: x = lo + c S + o with an integer cell c per axis
// (packed into `cell`, 10 bits per axis in 3D, 15 in 2D; bit 30 = clamped) and
// a float32 offset o in [0, S).  r_ij = (c_i - c_j) S + (o_i - o_j) is then
// accurate to float32 rounding of r itself in any box, with half the bytes of a
// split hi+lo position.  The deformation pass gathers RD (position, velocity,
// volume) and the momentum pass RM (position, M = P B0^T by columns, volume).
constexpr uint32_t kFixedBit = 1u << 30;

// Wendland gradient factor gs = (dW/dr)/r from d^2 (q = sqrt(d2)/h, no division).
__device__ __forceinline__ float gs_from_d2(float d2, const TLK<float>& K) {
    float q = d2 * rsqrtf(fmaxf(d2, 1e-30f)) * K.inv_h;
    float t = fmaf(-0.5f, q, 1.0f);
    return K.coef * t * t * t;
}

// me: the particle's RD record, whose first quarter (position code) and V0 equal the RM
// record's; given, the record's first 32-byte sector is written whole, so that L2 need not
// fetch the rest of it from DRAM before writing it back.
template <int DIM>
__device__ __forceinline__ void store_M(float* RM, int64_t i, const float* m, const F8* me = nullptr) {
    if (DIM == 2) {
        if (me) *reinterpret_cast<float4*>(RM + 8 * i) = make_float4(me->v[0], me->v[1], me->v[2], me->v[3]);
        *reinterpret_cast<float4*>(RM + 8 * i + 4) = make_float4(m[0], m[2], m[1], m[3]);
    } else {
        float* rec = RM + 16 * i;
        if (me) {
            *reinterpret_cast<float4*>(rec) = make_float4(me->v[0], me->v[1], me->v[2], me->v[3]);
            *reinterpret_cast<float4*>(rec + 4) = make_float4(m[0], m[3], m[6], me->v[7]);
        } else {
            rec[4] = m[0]; rec[5] = m[3]; rec[6] = m[6];
        }
        *reinterpret_cast<float4*>(rec + 8) = make_float4(m[1], m[4], m[7], 0.0f);
        *reinterpret_cast<float4*>(rec + 12) = make_float4(m[2], m[5], m[8], 0.0f);
    }
}

template <int DIM>
__global__ void k_tl_stress32(const float* __restrict__ H, const float* __restrict__ B0, int64_t n, TLK<float> K,
                              float* __restrict__ RM) {
    constexpr int NS = DIM == 2 ? 3 : 6;
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float h[DIM * DIM], b[NS], m[DIM * DIM];
    for (int k = 0; k < DIM * DIM; ++k) h[k] = H[k * n + i];
    for (int s = 0; s < NS; ++s) b[s] = B0[s * n + i];
    stress_factor<DIM, float>(h, b, K, m);
    store_M<DIM>(RM, i, m);
}

// One momentum pair (Eq. 30) from the neighbour's RM chunks: accumulates
// (M_i + M_j) grad0 W_ij V0_j, rows 0-1 paired and row 2 alone.
template <int DIM, bool PER>
__device__ __forceinline__ void mom_pair(float4 c0, float4 c1, float4 c2, float4 c3, const float* oi, uint32_t bi,
                                         const float2* mi01, const float* mi2, const TLK<float>& K,
                                         Kahan2& acc01, Kahan<float>& acc2) {
    float oj[DIM], r[DIM], d2;
    uint32_t bj;
    float Vj;
    if (DIM == 3) {
        oj[0] = c0.x; oj[1] = c0.y; oj[DIM - 1] = c0.z;
        bj = __float_as_uint(c0.w);
        Vj = c1.w;
    } else {
        oj[0] = c0.x; oj[1] = c0.y;
        bj = __float_as_uint(c0.z);
        Vj = c0.w;
    }
    rel_pair<DIM, PER>(oi, bi, oj, bj, K.ncell, K.S, K.Sl, K.periodic, r, d2);
    float gs = gs_from_d2(d2, K) * Vj;
    if (DIM == 2) {
        float2 s0 = __fadd2_rn(mi01[0], make_float2(c1.x, c1.y));
        float2 s1 = __fadd2_rn(mi01[1], make_float2(c1.z, c1.w));
        float g0 = gs * r[0], g1 = gs * r[1];
        acc01.add(__ffma2_rn(s1, make_float2(g1, g1), __fmul2_rn(s0, make_float2(g0, g0))));
    } else {
        float g0 = gs * r[0], g1 = gs * r[1], g2 = gs * r[DIM - 1];
        float2 s0 = __fadd2_rn(mi01[0], make_float2(c1.x, c1.y));
        float2 s1 = __fadd2_rn(mi01[1], make_float2(c2.x, c2.y));
        float2 s2 = __fadd2_rn(mi01[DIM - 1], make_float2(c3.x, c3.y));
        float2 t01 = __ffma2_rn(s2, make_float2(g2, g2),
                                __ffma2_rn(s1, make_float2(g1, g1), __fmul2_rn(s0, make_float2(g0, g0))));
        float t2 = fmaf(mi2[2] + c3.z, g2, fmaf(mi2[1] + c2.z, g1, (mi2[0] + c1.z) * g0));
        acc01.add(t01);
        acc2.add(t2);
    }
}

// One deformation-rate pair (Eq. 31) from the neighbour's RD chunks: accumulates
// V0_j (v_j - v_i) (x) grad0 W_ij column by column.
template <int DIM, bool PER>
__device__ __forceinline__ void defo_pair(float4 c0, float4 c1, const float* oi, uint32_t bi, float2 nv01, float nv2,
                                          const TLK<float>& K, Kahan2* c01, Kahan2& r2, Kahan<float>& l22) {
    float oj[DIM], r[DIM], d2;
    uint32_t bj;
    float w;
    if (DIM == 3) {
        oj[0] = c0.x; oj[1] = c0.y; oj[DIM - 1] = c0.z;
        bj = __float_as_uint(c0.w);
        w = c1.w;
    } else {
        oj[0] = c0.x; oj[1] = c0.y;
        bj = __float_as_uint(c0.z);
        w = c0.w;
    }
    rel_pair<DIM, PER>(oi, bi, oj, bj, K.ncell, K.S, K.Sl, K.periodic, r, d2);
    float gs = gs_from_d2(d2, K);
    float2 dv01 = __fmul2_rn(make_float2(w, w), __fadd2_rn(make_float2(c1.x, c1.y), nv01));
    if (DIM == 2) {
        c01[0].add(__fmul2_rn(dv01, make_float2(gs * r[0], gs * r[0])));
        c01[1].add(__fmul2_rn(dv01, make_float2(gs * r[1], gs * r[1])));
    } else {
        float g0 = gs * r[0], g1 = gs * r[1], g2 = gs * r[DIM - 1];
        float dv2 = w * (c1.z + nv2);
        c01[0].add(__fmul2_rn(dv01, make_float2(g0, g0)));
        c01[1].add(__fmul2_rn(dv01, make_float2(g1, g1)));
        c01[DIM - 1].add(__fmul2_rn(dv01, make_float2(g2, g2)));
        r2.add(__fmul2_rn(make_float2(dv2, dv2), make_float2(g0, g1)));
        l22.add(dv2 * g2);
    }
}

// Position relative to a reference cell, from an encoded record (offset o, cell bits):
// x = (c - c_ref) S + o, S split as Sh + Sl as in rel_pair.  Non-periodic boxes only
// (a periodic axis needs the pair's own minimum image, rel_pair).
template <int DIM>
__device__ __forceinline__ void rel_to_ref(const float* o, uint32_t b, uint32_t bref, const TLK<float>& K, float* x) {
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
        const float fdc = rel_cell_f<DIM>(b, a) - rel_cell_f<DIM>(bref, a);
        x[a] = fmaf(fdc, K.S[a], fmaf(fdc, K.Sl[a], o[a]));
    }
}

// One deformation-rate pair from tile-relative positions: xj = (x, y, z, V0_j) and
// vj = (v_x, v_y, v_z, .) of the neighbour; the same sum as defo_pair.
template <int DIM>
__device__ __forceinline__ void defo_pair_rel(float4 xj, float4 vj, const float* xi, float2 nv01, float nv2,
                                              const TLK<float>& K, Kahan2* c01, Kahan2& r2, Kahan<float>& l22) {
    float r[DIM];
    r[0] = xi[0] - xj.x;
    r[1] = xi[1] - xj.y;
    if (DIM == 3) r[DIM - 1] = xi[DIM - 1] - xj.z;
    float d2 = r[0] * r[0];
#pragma unroll
    for (int a = 1; a < DIM; ++a) d2 = fmaf(r[a], r[a], d2);
    const float gs = gs_from_d2(d2, K);
    const float w = xj.w;
    float2 dv01 = __fmul2_rn(make_float2(w, w), __fadd2_rn(make_float2(vj.x, vj.y), nv01));
    if (DIM == 2) {
        c01[0].add(__fmul2_rn(dv01, make_float2(gs * r[0], gs * r[0])));
        c01[1].add(__fmul2_rn(dv01, make_float2(gs * r[1], gs * r[1])));
    } else {
        float g0 = gs * r[0], g1 = gs * r[1], g2 = gs * r[DIM - 1];
        float dv2 = w * (vj.z + nv2);
        c01[0].add(__fmul2_rn(dv01, make_float2(g0, g0)));
        c01[1].add(__fmul2_rn(dv01, make_float2(g1, g1)));
        c01[DIM - 1].add(__fmul2_rn(dv01, make_float2(g2, g2)));
        r2.add(__fmul2_rn(make_float2(dv2, dv2), make_float2(g0, g1)));
        l22.add(dv2 * g2);
    }
}

// The products one deformation-rate pair adds (as defo_pair_rel): columns (L0c, L1c) of
// V0_j (v_j - v_i) (x) g_ij, (L20, L21) and L22.  FUSE adds them to `t` with one rounding
// each (a block of two pairs is summed first and enters the compensated sums once).
struct DefoTerms {
    float2 c[3];
    float2 r2;
    float l22;
};

template <int DIM, bool FUSE>
__device__ __forceinline__ void defo_terms_rel(float4 xj, float4 vj, const float* xi, float2 nv01, float nv2,
                                               const TLK<float>& K, DefoTerms& t) {
    float r[DIM];
    r[0] = xi[0] - xj.x;
    r[1] = xi[1] - xj.y;
    if (DIM == 3) r[DIM - 1] = xi[DIM - 1] - xj.z;
    float d2 = r[0] * r[0];
#pragma unroll
    for (int a = 1; a < DIM; ++a) d2 = fmaf(r[a], r[a], d2);
    const float gs = gs_from_d2(d2, K);
    const float w = xj.w;
    const float2 dv01 = __fmul2_rn(make_float2(w, w), __fadd2_rn(make_float2(vj.x, vj.y), nv01));
    const float g0 = gs * r[0], g1 = gs * r[1];
    if (FUSE) {
        t.c[0] = __ffma2_rn(dv01, make_float2(g0, g0), t.c[0]);
        t.c[1] = __ffma2_rn(dv01, make_float2(g1, g1), t.c[1]);
    } else {
        t.c[0] = __fmul2_rn(dv01, make_float2(g0, g0));
        t.c[1] = __fmul2_rn(dv01, make_float2(g1, g1));
    }
    if (DIM == 3) {
        const float g2 = gs * r[DIM - 1];
        const float dv2 = w * (vj.z + nv2);
        if (FUSE) {
            t.c[DIM - 1] = __ffma2_rn(dv01, make_float2(g2, g2), t.c[DIM - 1]);
            t.r2 = __ffma2_rn(make_float2(dv2, dv2), make_float2(g0, g1), t.r2);
            t.l22 = fmaf(dv2, g2, t.l22);
        } else {
            t.c[DIM - 1] = __fmul2_rn(dv01, make_float2(g2, g2));
            t.r2 = __fmul2_rn(make_float2(dv2, dv2), make_float2(g0, g1));
            t.l22 = dv2 * g2;
        }
    }
}

template <int DIM>
__device__ __forceinline__ void defo_add_terms(const DefoTerms& t, Kahan2* c01, Kahan2& r2, Kahan<float>& l22) {
    c01[0].add(t.c[0]);
    c01[1].add(t.c[1]);
    if (DIM == 3) {
        c01[DIM - 1].add(t.c[DIM - 1]);
        r2.add(t.r2);
        l22.add(t.l22);
    }
}

__device__ __forceinline__ float4 lo4(const F8& f) { return make_float4(f.v[0], f.v[1], f.v[2], f.v[3]); }
__device__ __forceinline__ float4 hi4(const F8& f) { return make_float4(f.v[4], f.v[5], f.v[6], f.v[7]); }

// Own stress factor M_i by columns from the RM record (rows 0-1 paired, row 2 alone).
template <int DIM>
__device__ __forceinline__ void own_M(const F8& a0, const F8& a1, float2* mi01, float* mi2) {
    if (DIM == 2) {
        mi01[0] = make_float2(a0.v[4], a0.v[5]);
        mi01[1] = make_float2(a0.v[6], a0.v[7]);
    } else {
        mi01[0] = make_float2(a0.v[4], a0.v[5]); mi2[0] = a0.v[6];
        mi01[1] = make_float2(a1.v[0], a1.v[1]); mi2[1] = a1.v[2];
        mi01[DIM - 1] = make_float2(a1.v[4], a1.v[5]); mi2[2] = a1.v[6];
    }
}

// Momentum pass (Eq. 30), neighbours gathered from global memory (states without
// a tile plan).  LANES lanes per row; the next neighbour's record is loaded before
// the current pair is evaluated.
template <int DIM, int OUT, int LANES, bool PER>
__global__ void __launch_bounds__(256, 4) k_tl_mom32(const float* __restrict__ RM, float* __restrict__ RD,
                                                     const int64_t* __restrict__ row_ptr,
                                                     const int32_t* __restrict__ col, int64_t n, TLK<float> K,
                                                     double* __restrict__ dvdt) {
    constexpr int W = DIM == 3 ? 16 : 8;
    int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t i = gt / LANES;
    int lane = (int)(gt % LANES);
    bool active = i < n;
    int64_t ii = active ? i : 0;
    F8 a0 = ldg8(RM + W * ii);
    F8 a1 = DIM == 3 ? ldg8(RM + W * ii + 8) : a0;
    float oi[DIM];
#pragma unroll
    for (int a = 0; a < DIM; ++a) oi[a] = a0.v[a];
    uint32_t bi = __float_as_uint(a0.v[DIM]);
    float2 mi01[DIM];
    float mi2[3] = {0.0f, 0.0f, 0.0f};
    own_M<DIM>(a0, a1, mi01, mi2);
    Kahan2 acc01;
    Kahan<float> acc2;
    acc01.init();
    acc2.init();
    int64_t b = active ? row_ptr[ii] : 0, e = active ? row_ptr[ii + 1] : 0;
    int64_t p = b + lane;
    int j = p < e ? __ldg(&col[p]) : -1;
    F8 r0 = a0, r1 = a1;
    if (j >= 0) {
        r0 = ldg8(RM + W * (int64_t)j);
        if (DIM == 3) r1 = ldg8(RM + W * (int64_t)j + 8);
    }
    while (j >= 0) {
        int64_t pn = p + LANES;
        int jn = pn < e ? __ldg(&col[pn]) : -1;
        F8 n0 = r0, n1 = r1;
        if (jn >= 0) {
            n0 = ldg8(RM + W * (int64_t)jn);
            if (DIM == 3) n1 = ldg8(RM + W * (int64_t)jn + 8);
        }
        mom_pair<DIM, PER>(lo4(r0), hi4(r0), lo4(r1), hi4(r1), oi, bi, mi01, mi2, K, acc01, acc2);
        p = pn;
        j = jn;
        r0 = n0;
        r1 = n1;
    }
    float2 v01 = acc01.value();
    float tot[3] = {group_sum<LANES>(v01.x), group_sum<LANES>(v01.y), 0.0f};
    if (DIM == 3) tot[2] = group_sum<LANES>(acc2.value());
    if (!active || lane != 0) return;
    if (OUT == OUT_RATES) {
        for (int a = 0; a < DIM; ++a) dvdt[a * n + i] = (double)(tot[a] * K.inv_rho0);
        return;
    }
    bool fx = (bi & kFixedBit) != 0;
    float* vrec = RD + 8 * i + 4;
#pragma unroll
    for (int a = 0; a < DIM; ++a) vrec[a] = fx ? 0.0f : vrec[a] + K.dt * (tot[a] * K.inv_rho0);
}

// Deformation-rate epilogue shared by both forms of the pass: F_i += dt L B0_i
// (F = I on clamped particles), x_i += dt v_i and the next step's M_i = P(F_i) B0_i^T.
// hold/uold: the row's current H and u when already loaded (else read here).  Hx/ux: a
// second copy of the new H and u (the caller's mapped host arrays), written beside H, u.
template <int DIM, int OUT>
__device__ __forceinline__ void defo_finish(const float* Lt, const float* b0, bool fx, const float* vi, int64_t i,
                                            int64_t n, const TLK<float>& K, float* __restrict__ RM,
                                            float* __restrict__ H, float* __restrict__ u,
                                            double* __restrict__ dFdt, const float* hold = nullptr,
                                            const float* uold = nullptr, const F8* me = nullptr,
                                            float* __restrict__ Hx = nullptr, float* __restrict__ ux = nullptr) {
    float Fd[DIM * DIM];
    times_b0<DIM, float>(Lt, b0, Fd);
    if (OUT == OUT_RATES) {
        for (int k = 0; k < DIM * DIM; ++k) dFdt[k * n + i] = (double)Fd[k];
        return;
    }
    float h[DIM * DIM], m[DIM * DIM];
#pragma unroll
    for (int k = 0; k < DIM * DIM; ++k) {
        h[k] = fx ? 0.0f : (hold ? hold[k] : H[k * n + i]) + K.dt * Fd[k];
        H[k * n + i] = h[k];
        if (Hx) Hx[k * n + i] = h[k];
    }
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
        const float ua = (uold ? uold[a] : u[a * n + i]) + K.dt * vi[a];
        u[a * n + i] = ua;
        if (ux) ux[a * n + i] = ua;
    }
    stress_factor<DIM, float>(h, b0, K, m);
    store_M<DIM>(RM, i, m, me);
}

// Deformation-rate pass (Eq. 31) with the fused stress update of the next step,
// neighbours gathered from global memory.  L = sum_j V0_j (v_j - v_i) (x) g_ij is
// accumulated column by column: rows 0-1 of each column in one paired compensated
// accumulator, row 2 of columns 0-1 in a second pair and L22 in a scalar one.
template <int DIM, int OUT, int LANES, bool PER>
__global__ void __launch_bounds__(256, 4) k_tl_defo32(const float* __restrict__ RD, float* __restrict__ RM,
                                                      const int64_t* __restrict__ row_ptr,
                                                      const int32_t* __restrict__ col, int64_t n, TLK<float> K,
                                                      const float* __restrict__ B0, float* __restrict__ H,
                                                      float* __restrict__ u, double* __restrict__ dFdt) {
    constexpr int NS = DIM == 2 ? 3 : 6;
    int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t i = gt / LANES;
    int lane = (int)(gt % LANES);
    bool active = i < n;
    int64_t ii = active ? i : 0;
    F8 me = ldg8(RD + 8 * ii);
    float oi[DIM];
#pragma unroll
    for (int a = 0; a < DIM; ++a) oi[a] = me.v[a];
    uint32_t bi = __float_as_uint(me.v[DIM]);
    float2 nv01 = make_float2(-me.v[4], -me.v[5]);
    float nv2 = -me.v[6];
    Kahan2 c01[DIM];
    Kahan2 r2;
    Kahan<float> l22;
#pragma unroll
    for (int c = 0; c < DIM; ++c) c01[c].init();
    r2.init();
    l22.init();
    int64_t b = active ? row_ptr[ii] : 0, e = active ? row_ptr[ii + 1] : 0;
    int64_t p = b + lane;
    int j = p < e ? __ldg(&col[p]) : -1;
    F8 rj = me;
    if (j >= 0) rj = ldg8(RD + 8 * (int64_t)j);
    while (j >= 0) {
        int64_t pn = p + LANES;
        int jn = pn < e ? __ldg(&col[pn]) : -1;
        F8 rn = rj;
        if (jn >= 0) rn = ldg8(RD + 8 * (int64_t)jn);
        defo_pair<DIM, PER>(lo4(rj), hi4(rj), oi, bi, nv01, nv2, K, c01, r2, l22);
        p = pn;
        j = jn;
        rj = rn;
    }
    float Lt[DIM * DIM];
#pragma unroll
    for (int c = 0; c < DIM; ++c) {
        float2 v = c01[c].value();
        Lt[0 * DIM + c] = group_sum<LANES>(v.x);
        Lt[1 * DIM + c] = group_sum<LANES>(v.y);
    }
    if (DIM == 3) {
        float2 v = r2.value();
        Lt[2 * DIM + 0] = group_sum<LANES>(v.x);
        Lt[2 * DIM + 1] = group_sum<LANES>(v.y);
        Lt[2 * DIM + 2] = group_sum<LANES>(l22.value());
    }
    if (!active || lane != 0) return;
    float b0[NS], vi[3] = {me.v[4], me.v[5], me.v[6]};
#pragma unroll
    for (int s = 0; s < NS; ++s) b0[s] = B0[s * n + i];
    defo_finish<DIM, OUT>(Lt, b0, (bi & kFixedBit) != 0, vi, i, n, K, RM, H, u, dFdt, nullptr, nullptr, &me);
}

// ------------------------------------------------ float32 passes on a tile plan
// With a tile plan (tiles.cuh) the pair geometry of the fixed reference
// configuration is computed once, in float64, by k_tl_geo: entry (k, r) of tile b
// holds w = grad0 W_ij V0_j (rounded to float32) and, in .w, the position of j among
// the tile's distinct neighbours.  A block is one tile, one thread per row: it
// stages the neighbours' M_j (momentum) or v_j (deformation) in shared memory and
// its warps read the pair entries 512 contiguous bytes at a time.
// Polls of a bounded mbarrier wait before a block gives up (FLAG_TIMEOUT).
constexpr uint32_t kWaitPolls = 1u << 22;

struct GeoArgs {
    const int32_t* tile_m;
    const int64_t* tile_so;
    const int32_t* uidx;
    const float4* geo;
    int mcap;
    const int32_t* tile_e;   // bulk form: entries per tile
    int ecap;                // bulk form: most entries a block copies into shared memory (0: none)
    const uint16_t* slots;   // geometry form: the pairs' staging positions alone, same sliced order
    const float4* wsum;      // geometry form of the momentum pass: (S_i, 0) per particle
    const uint16_t* spos;    // geometry form: staging position of each distinct neighbour (uidx order)
    const uint16_t* sinv;    // geometry form: the distinct neighbour at each staging position
    uint32_t test_polls;     // bulk form: > 0 issues no copy and waits this many polls (sph_set_wait_test)
};

// The TL plan: the tile plan (tiles.cuh) with 16-byte entries, then the entries' slots
// alone as a sliced uint16 section (read by the passes that evaluate the pair geometry
// from the staged records instead of reading the entries), then per particle the float4
// (S_i, 0) with S_i = sum_j grad0 W_ij V0_j, a fixed property of the reference
// configuration that the geometry form of the momentum pass uses.
static inline size_t tl_slot_offset(int64_t n, int64_t nnz, int64_t maxrow) {
    return tile_plan_bytes(n, nnz, maxrow);
}

static inline size_t tl_wsum_offset(int64_t n, int64_t nnz, int64_t maxrow) {
    const int64_t ntiles = (n + kTileRows - 1) / kTileRows;
    return tl_slot_offset(n, nnz, maxrow) + align16((size_t)ntiles * kTileRows * (size_t)maxrow * 2);
}

// Then two uint16 sections indexed like uidx (tile b's k-th distinct neighbour at
// row_ptr[b * kTileRows] + k): spos, the shared-memory position the geometry-form passes
// stage that neighbour at, and sinv, its inverse (the neighbour at each position).
static inline size_t tl_spos_offset(int64_t n, int64_t nnz, int64_t maxrow) {
    return tl_wsum_offset(n, nnz, maxrow) + align16((size_t)n * 16);
}

static inline size_t tl_sinv_offset(int64_t n, int64_t nnz, int64_t maxrow) {
    return tl_spos_offset(n, nnz, maxrow) + align16((size_t)nnz * 2);
}

static inline size_t tl_plan_total(int64_t n, int64_t nnz, int64_t maxrow) {
    return tl_sinv_offset(n, nnz, maxrow) + align16((size_t)nnz * 2);
}

// Most distinct neighbours of a tile whose staging positions are balanced over the bank
// groups (tiles with more keep their list order).
constexpr int kPermCap = 2048;

// Pair order of a tile's rows for the staged 16-byte gathers of the geometry-form passes.
// The k-th pairs of a quarter warp's 8 rows (consecutive rows) are read by one gather, which
// takes one wavefront when its lanes read 8 different groups (position mod 8) and as many as
// the most lanes on one group otherwise.  Step by step, a maximum matching of the quarter's
// active rows to groups in which they have pairs left is found by augmenting paths (Kuhn):
// rows in order of most pairs left, each trying its groups in order of most of its pairs
// left in them (ties to the lower row, the lower group).  A row left unmatched takes the
// group picked least often so far in the step, then the one with most of its pairs left,
// then the lower group.  In a group a row takes its pairs in list order.  One thread per
// quarter warp computes the matchings; every thread of the block must call this (block
// barriers).  scratch: kTileRows * (kSortCap + 8) bytes of shared memory.  order[k] receives
// the list position of the row's k-th pair; rows longer than kSortCap keep list order, take
// no part, and get false.
template <typename SF>
__device__ __forceinline__ bool quarter_match_order(int len, SF slot_of, uint32_t* order, uint8_t* scratch) {
    const int row = (int)threadIdx.x;
    const bool fits = len <= kSortCap;
    const int my = fits ? len : 0;
    uint8_t* s_choice = scratch;                                   // [row][step]: the group read
    uint8_t* s_rem = scratch + kTileRows * kSortCap;               // [row][group]: pairs left
    // the row's pairs by group (a counting sort of list positions), in list order within one
    uint8_t byg[kSortCap];
    int cnt[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int k = 0; k < my; ++k) {
        const int g = slot_of(k) & 7;
#pragma unroll
        for (int c = 0; c < 8; ++c) cnt[c] += c == g ? 1 : 0;
    }
#pragma unroll
    for (int g = 0; g < 8; ++g) s_rem[8 * row + g] = (uint8_t)cnt[g];
    __syncthreads();
    if ((row & 7) == 0) {
        // one thread per quarter warp; its state in packed registers: owner (group -> row),
        // mg (row -> group) and picks (group -> count) as 4-bit fields, left (row -> pairs
        // left) as 8-bit fields, the search stack as 4-bit fields
        const int r0 = row;
        const uint8_t* rem = s_rem + 8 * r0;
        uint64_t left = 0u;
        int steps = 0;
        for (int r = 0; r < 8; ++r) {
            int l = 0;
            for (int g = 0; g < 8; ++g) l += rem[8 * r + g];
            left |= (uint64_t)l << (8 * r);
            steps = max(steps, l);
        }
        auto lft = [&](int r) { return (int)((left >> (8 * r)) & 0xFFu); };
        for (int p = 0; p < steps; ++p) {
            uint32_t owner = 0x88888888u, mg = 0x88888888u;
            uint32_t done = 0u;                                    // rows already taken this step
            for (;;) {
                // the next row: most pairs left, then the lower row
                int rs = -1, ls = 0;
                for (int r = 0; r < 8; ++r) {
                    const int l = lft(r);
                    if (((done >> r) & 1u) == 0u && l > ls) {
                        rs = r;
                        ls = l;
                    }
                }
                if (rs < 0) break;
                done |= 1u << rs;
                // augmenting path from rs, depth first; at a row the unseen group with most of
                // its pairs left, then the lower group; each group seen once per search
                uint64_t st_r = (uint64_t)rs, st_g = 0u;
                int depth = 0;
                uint32_t seen = 0u;
                while (depth >= 0) {
                    const int r = (int)((st_r >> (4 * depth)) & 15u);
                    int best = -1, bc = 0;
                    for (int g = 0; g < 8; ++g) {
                        const int c = rem[8 * r + g];
                        if (((seen >> g) & 1u) == 0u && c > bc) {
                            best = g;
                            bc = c;
                        }
                    }
                    if (best < 0) {
                        --depth;
                        continue;
                    }
                    seen |= 1u << best;
                    st_g = (st_g & ~(15ull << (4 * depth))) | ((uint64_t)best << (4 * depth));
                    const int ow = (int)((owner >> (4 * best)) & 15u);
                    if (ow == 8) {
                        for (int d = 0; d <= depth; ++d) {
                            const int gd = (int)((st_g >> (4 * d)) & 15u), rd = (int)((st_r >> (4 * d)) & 15u);
                            owner = (owner & ~(15u << (4 * gd))) | ((uint32_t)rd << (4 * gd));
                            mg = (mg & ~(15u << (4 * rd))) | ((uint32_t)gd << (4 * rd));
                        }
                        break;
                    }
                    if (depth >= 7) continue;                      // never: 8 groups bound the depth
                    ++depth;
                    st_r = (st_r & ~(15ull << (4 * depth))) | ((uint64_t)ow << (4 * depth));
                }
            }
            uint32_t picks = 0u;
            for (int g = 0; g < 8; ++g) picks |= (((owner >> (4 * g)) & 15u) != 8u ? 1u : 0u) << (4 * g);
            // rows left unmatched, in the same order: the group picked least often, then the
            // one with most of the row's pairs left, then the lower group
            done = 0u;
            for (;;) {
                int rs = -1, ls = 0;
                for (int r = 0; r < 8; ++r) {
                    const int l = lft(r);
                    if (((done >> r) & 1u) == 0u && l > ls) {
                        rs = r;
                        ls = l;
                    }
                }
                if (rs < 0) break;
                done |= 1u << rs;
                if (((mg >> (4 * rs)) & 15u) != 8u) continue;
                int best = -1;
                for (int g = 0; g < 8; ++g) {
                    const int c = rem[8 * rs + g];
                    if (c == 0) continue;
                    const int pk = (int)((picks >> (4 * g)) & 15u);
                    const int pb = best < 0 ? 0 : (int)((picks >> (4 * best)) & 15u);
                    if (best < 0 || pk < pb || (pk == pb && c > rem[8 * rs + best])) best = g;
                }
                mg = (mg & ~(15u << (4 * rs))) | ((uint32_t)best << (4 * rs));
                picks += 1u << (4 * best);
            }
            for (int r = 0; r < 8; ++r) {
                if (lft(r) == 0) continue;
                const int g = (int)((mg >> (4 * r)) & 15u);
                s_choice[(r0 + r) * kSortCap + p] = (uint8_t)g;
                s_rem[8 * (r0 + r) + g] -= 1;
                left -= 1ull << (8 * r);
            }
        }
    }
    __syncthreads();
    // the row's pairs by group, list order within a group, then the chosen groups in turn
    int start[8];
    {
        int acc = 0;
#pragma unroll
        for (int g = 0; g < 8; ++g) {
            start[g] = acc;
            acc += cnt[g];
        }
    }
    for (int k = 0; k < my; ++k) {
        const int g = slot_of(k) & 7;
        int at = 0;
#pragma unroll
        for (int c = 0; c < 8; ++c)
            if (c == g) at = start[c]++;
        byg[at] = (uint8_t)k;
    }
#pragma unroll
    for (int g = 7; g >= 0; --g) start[g] = g == 0 ? 0 : start[g - 1];   // back to the first of each group
    for (int p = 0; p < my; ++p) {
        const int g = s_choice[row * kSortCap + p];
        int at = 0;
#pragma unroll
        for (int c = 0; c < 8; ++c)
            if (c == g) at = start[c]++;
        order[p] = (uint32_t)byg[min(at, my - 1)];
    }
    return fits;
}

// Pair entries of the tile plan: w = grad0 W_ij V0_j in float64, stored float32,
// with the neighbour's slot (its position in the tile's distinct list); the row's
// S_i = sum_j w_ij, summed in float64 in list order, stored float32; and the staging
// positions of the geometry forms.
//
// Staging positions: a quarter warp's 16-byte shared-memory gathers take one wavefront
// when its 8 lanes read positions in 8 different groups (position mod 8), so the tile's
// distinct neighbours are given positions whose groups balance, in every quarter warp
// (8 consecutive rows), the pairs over the 8 groups.  Greedily, in list order: each
// neighbour takes the group with room (group c holds the positions c, c + 8, ... below
// m) that adds least to sum over quarter warps and groups of (pairs in the group)^2,
// i.e. the smallest sum_Q cnt_Q * load_Q[c], ties to the lower group, among the groups
// not yet taken in its aligned block of 8 consecutive neighbours (any group with room
// when none is left).  The staging loops store 8 consecutive neighbours per quarter
// warp, so their 16-byte stores fall in 8 different groups, while their loads follow
// the column order.  Each row's pairs are then laid out in the bank-aware order
// (bank_order) of these positions.
template <int DIM>
__global__ void __launch_bounds__(kTileRows) k_tl_geo(const double* __restrict__ r0, const double* __restrict__ V0,
                                                      const int64_t* __restrict__ row_ptr,
                                                      const int32_t* __restrict__ col,
                                                      const uint16_t* __restrict__ lcol,
                                                      const int32_t* __restrict__ tile_m,
                                                      const int32_t* __restrict__ tile_e,
                                                      const int64_t* __restrict__ tile_so, int64_t n, TLK<double> K,
                                                      float4* __restrict__ geo, uint16_t* __restrict__ slots,
                                                      float4* __restrict__ wsum, uint16_t* __restrict__ spos,
                                                      uint16_t* __restrict__ sinv) {
    __shared__ uint32_t s_cnt[kPermCap * 4];   // per neighbour, the 16 quarter warps' pair counts, a byte each
    __shared__ uint16_t s_pos[kPermCap];
    __shared__ int s_load[16 * 8];
    __shared__ int s_used[8];
    const int64_t tile = blockIdx.x;
    const int64_t i = tile * kTileRows + threadIdx.x;
    const bool active = i < n;
    const int64_t b = active ? row_ptr[i] : 0;
    const int len = active ? (int)(row_ptr[i + 1] - b) : 0;
    const int width = tile_e[tile] / kTileRows;
    const int m = tile_m[tile];
    const int64_t P0 = row_ptr[tile * kTileRows];
    float4* out = geo + tile_so[tile] + threadIdx.x;
    double xi[DIM];
#pragma unroll
    for (int a = 0; a < DIM; ++a) xi[a] = active ? r0[a * n + i] : 0.0;
    const bool balance = m <= kPermCap;
    if (balance) {
        for (int q = threadIdx.x; q < 4 * m; q += blockDim.x) s_cnt[q] = 0u;
        for (int q = threadIdx.x; q < 16 * 8; q += blockDim.x) s_load[q] = 0;
        if (threadIdx.x < 8) s_used[threadIdx.x] = 0;
        __syncthreads();
        const int Q = (int)threadIdx.x >> 3;
        for (int k = 0; k < len; ++k)
            atomicAdd(&s_cnt[4 * min((int)lcol[b + k], m - 1) + (Q >> 2)], 1u << (8 * (Q & 3)));
        __syncthreads();
        if (threadIdx.x < 32) {
            const int lane = (int)threadIdx.x;
            uint32_t block_used = 0u;      // groups taken in the current aligned block of 8 neighbours
            for (int q = 0; q < m; ++q) {
                uint32_t key = 0xFFFFFFFFu;
                if (lane < 8 && s_used[lane] < (m - lane + 7) / 8) {
                    uint32_t cost = 0u;
#pragma unroll
                    for (int qi = 0; qi < 16; ++qi)
                        cost += ((s_cnt[4 * q + (qi >> 2)] >> (8 * (qi & 3))) & 0xFFu) * (uint32_t)s_load[8 * qi + lane];
                    key = (((block_used >> lane) & 1u) << 31) | (cost * 8u + (uint32_t)lane);
                }
                const int c = (int)(__reduce_min_sync(0xFFFFFFFFu, key) & 7u);
                block_used = (q & 7) == 7 ? 0u : (block_used | (1u << c));
                if (lane < 16) s_load[8 * lane + c] += (int)((s_cnt[4 * q + (lane >> 2)] >> (8 * (lane & 3))) & 0xFFu);
                __syncwarp();
                if (lane == 0) {
                    s_pos[q] = (uint16_t)c;          // the group; positions follow the refinement
                    s_used[c] += 1;
                }
                __syncwarp();
            }
            // refinement: two neighbours of one aligned block exchange their groups when that
            // lowers the sum over quarter warps and groups of load^2 (the block keeps its
            // groups, each group its size), for at most three sweeps over the blocks
            for (int sweep = 0; sweep < 3; ++sweep) {
                bool changed = false;
                for (int b0 = 0; b0 < m; b0 += 8) {
                    const int bn = min(8, m - b0);
                    for (int x = 0; x < bn; ++x)
                        for (int y = x + 1; y < bn; ++y) {
                            const int qa = b0 + x, qb = b0 + y;
                            const int ga = s_pos[qa], gb = s_pos[qb];
                            if (ga == gb) continue;
                            int d = 0, delta = 0;
                            if (lane < 16) {
                                const int sh = 8 * (lane & 3);
                                d = (int)((s_cnt[4 * qa + (lane >> 2)] >> sh) & 0xFFu) -
                                    (int)((s_cnt[4 * qb + (lane >> 2)] >> sh) & 0xFFu);
                                // (l_a - d)^2 + (l_b + d)^2 - l_a^2 - l_b^2
                                delta = 2 * d * (s_load[8 * lane + gb] - s_load[8 * lane + ga] + d);
                            }
                            delta = __reduce_add_sync(0xFFFFFFFFu, delta);
                            if (delta < 0) {
                                if (lane < 16) {
                                    s_load[8 * lane + ga] -= d;
                                    s_load[8 * lane + gb] += d;
                                }
                                if (lane == 0) {
                                    s_pos[qa] = (uint16_t)gb;
                                    s_pos[qb] = (uint16_t)ga;
                                }
                                changed = true;
                            }
                            __syncwarp();
                        }
                }
                if (!changed) break;
            }
            // positions: within its group, a neighbour's rank in list order
            if (lane == 0) {
                int rank[8] = {0, 0, 0, 0, 0, 0, 0, 0};
                for (int q = 0; q < m; ++q) {
                    const int c = s_pos[q] & 7;
                    s_pos[q] = (uint16_t)(8 * rank[c] + c);
                    rank[c] += 1;
                }
            }
        }
        __syncthreads();
        for (int q = threadIdx.x; q < m; q += blockDim.x) {
            spos[P0 + q] = s_pos[q];
            sinv[P0 + s_pos[q]] = (uint16_t)q;
        }
    } else {
        for (int q = threadIdx.x; q < m; q += blockDim.x) {
            spos[P0 + q] = (uint16_t)q;
            sinv[P0 + q] = (uint16_t)q;
        }
    }
    auto pos_of = [&](int q) { return balance ? (int)s_pos[min(q, m - 1)] : q; };
    // pair order for the staged 16-byte gathers (see quarter_match_order); its tables reuse
    // s_cnt, free once the positions are set
    __syncthreads();
    uint32_t order[kSortCap];
    const bool sorted = quarter_match_order(len, [&](int k) { return pos_of((int)lcol[b + k]); }, order,
                                            reinterpret_cast<uint8_t*>(s_cnt));
    for (int k = 0; k < width; ++k) {
        float4 e = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        if (k < len) {
            int64_t p = b + (sorted ? (int)(order[k] & 0xFFFFFu) : k);
            int j = col[p];
            double r[DIM], d2;
            pair_r64<DIM>(xi, r0, n, j, K, r, d2);
            double gv = wendland_gs<double>(sqrt(d2) * K.inv_h, K.coef) * V0[j];
            e.x = (float)(gv * r[0]);
            e.y = (float)(gv * r[1]);
            if (DIM == 3) e.z = (float)(gv * r[DIM - 1]);
            e.w = __int_as_float((int)lcol[p]);
        }
        out[(int64_t)k * kTileRows] = e;
        slots[tile_so[tile] + threadIdx.x + (int64_t)k * kTileRows] =
            k < len ? (uint16_t)pos_of(__float_as_int(e.w)) : (uint16_t)0;
    }
    if (!active) return;
    double S[3] = {0.0, 0.0, 0.0};
    for (int k = 0; k < len; ++k) {
        int j = col[b + k];
        double r[DIM], d2;
        pair_r64<DIM>(xi, r0, n, j, K, r, d2);
        double gv = wendland_gs<double>(sqrt(d2) * K.inv_h, K.coef) * V0[j];
#pragma unroll
        for (int a = 0; a < DIM; ++a) S[a] += gv * r[a];
    }
    wsum[i] = make_float4((float)S[0], (float)S[1], (float)S[2], 0.0f);
}

// Stage chunks FIRST..FIRST+NPL-1 of the tile's distinct neighbours' records (record
// stride RECF floats) at sp[c * mcap + s].  Returns false, staging nothing, for a tile
// with more distinct neighbours than mcap.  Block-uniform.
template <int NPL, int RECF, int FIRST = 1>
__device__ __forceinline__ bool stage_neighbours(const float* __restrict__ R, int64_t n, int64_t P0, int m,
                                                 const GeoArgs& A, float4* sp, const uint16_t* spos = nullptr) {
    const bool staged = m <= A.mcap;
    if (staged) {
        // consecutive threads copy consecutive chunks of consecutive neighbours: the
        // tile's neighbours come in runs of consecutive indices (Morton order), so the
        // loads of a warp mostly fall on contiguous records.  spos: the staging position
        // of each neighbour (else its place in the list)
        for (int q = threadIdx.x; q < m * NPL; q += blockDim.x) {
            int s = q / NPL, c = q - s * NPL;
            // a plan out of date with the lists reads wrong but in-bounds records
            int64_t j = min(max((int64_t)A.uidx[P0 + s], (int64_t)0), n - 1);
            const int at = spos ? min((int)spos[P0 + s], m - 1) : s;
            sp[c * A.mcap + at] = __ldg(reinterpret_cast<const float4*>(R + RECF * j) + FIRST + c);
        }
    }
    __syncthreads();
    return staged;
}

template <int DIM, int OUT>
__global__ void __launch_bounds__(kTileRows, 7) k_tl_mom32g(const float* __restrict__ RM, float* __restrict__ RD,
                                                            const int64_t* __restrict__ row_ptr, int64_t n,
                                                            TLK<float> K, GeoArgs A, double* __restrict__ dvdt) {
    constexpr int W = DIM == 3 ? 16 : 8;
    constexpr int NPL = DIM == 3 ? 3 : 1;
    extern __shared__ __align__(16) unsigned char tl_smem[];
    float4* sp = reinterpret_cast<float4*>(tl_smem);
    // tiles in reverse: the deformation pass walks them forwards, so each pass starts on
    // the pair entries the previous one read last, still in L2
    const int64_t tile = gridDim.x - 1 - blockIdx.x;
    const int64_t i0 = tile * kTileRows;
    const int64_t i = i0 + threadIdx.x;
    const bool active = i < n;
    const int64_t ii = active ? i : i0;
    // own loads first: their latency overlaps the staging
    const int64_t P0 = row_ptr[i0];
    const int len = active ? (int)(row_ptr[ii + 1] - row_ptr[ii]) : 0;
    const int m = A.tile_m[tile];
    const float4* g = A.geo + A.tile_so[tile] + threadIdx.x;
    F8 a0 = ldg8(RM + W * ii);
    F8 a1 = DIM == 3 ? ldg8(RM + W * ii + 8) : a0;
    float vown[3] = {0.0f, 0.0f, 0.0f};
    if (OUT != OUT_RATES) {
#pragma unroll
        for (int a = 0; a < DIM; ++a) vown[a] = RD[8 * ii + 4 + a];
    }
    // 3D: each staged M_j as 9 floats, planes (M00, M10, M01, M11), (M02, M12, M20, M21)
    // and M22, three shared-memory loads of 36 bytes per pair; 2D: one chunk
    float* sp2 = reinterpret_cast<float*>(sp + 2 * A.mcap);
    bool staged;
    if (DIM == 3) {
        staged = m <= A.mcap;
        if (staged) {
            for (int q = threadIdx.x; q < m; q += blockDim.x) {
                // a plan out of date with the lists reads wrong but in-bounds records
                int64_t j = min(max((int64_t)A.uidx[P0 + q], (int64_t)0), n - 1);
                const float4* rec = reinterpret_cast<const float4*>(RM + W * j);
                float4 c1 = __ldg(rec + 1), c2 = __ldg(rec + 2), c3 = __ldg(rec + 3);
                sp[q] = make_float4(c1.x, c1.y, c2.x, c2.y);
                sp[A.mcap + q] = make_float4(c3.x, c3.y, c1.z, c2.z);
                sp2[q] = c3.z;
            }
        }
        __syncthreads();
    } else {
        staged = stage_neighbours<NPL, W>(RM, n, P0, m, A, sp);
    }
    const uint32_t bi = __float_as_uint(a0.v[DIM]);
    float2 mi01[DIM];
    float mi2[3] = {0.0f, 0.0f, 0.0f};
    own_M<DIM>(a0, a1, mi01, mi2);
    Kahan2 acc01;
    Kahan<float> acc2;
    acc01.init();
    acc2.init();
    auto pair = [&](float4 e, float4 c1, float4 c2, float4 c3) {
        if (DIM == 2) {
            float2 s0 = __fadd2_rn(mi01[0], make_float2(c1.x, c1.y));
            float2 s1 = __fadd2_rn(mi01[1], make_float2(c1.z, c1.w));
            acc01.add(__ffma2_rn(s1, make_float2(e.y, e.y), __fmul2_rn(s0, make_float2(e.x, e.x))));
        } else {
            float2 s0 = __fadd2_rn(mi01[0], make_float2(c1.x, c1.y));
            float2 s1 = __fadd2_rn(mi01[1], make_float2(c2.x, c2.y));
            float2 s2 = __fadd2_rn(mi01[DIM - 1], make_float2(c3.x, c3.y));
            float2 t01 = __ffma2_rn(s2, make_float2(e.z, e.z),
                                    __ffma2_rn(s1, make_float2(e.y, e.y), __fmul2_rn(s0, make_float2(e.x, e.x))));
            float t2 = fmaf(mi2[2] + c3.z, e.z, fmaf(mi2[1] + c2.z, e.y, (mi2[0] + c1.z) * e.x));
            acc01.add(t01);
            acc2.add(t2);
        }
    };
    const int mc = A.mcap;
    if (staged) {
#pragma unroll 4
        for (int k = 0; k < len; ++k) {
            float4 e = ldg4_stream(g + (int64_t)k * kTileRows);
            int s = min(max(__float_as_int(e.w), 0), max(m - 1, 0));
            if (DIM == 3) {
                const float4 p0 = sp[s], p1 = sp[mc + s];
                const float m22 = sp2[s];
                // the record chunks (M00, M10, M20, .) (M01, M11, M21, .) (M02, M12, M22, .)
                pair(e, make_float4(p0.x, p0.y, p1.z, 0.0f), make_float4(p0.z, p0.w, p1.w, 0.0f),
                     make_float4(p1.x, p1.y, m22, 0.0f));
            } else {
                float4 c1 = sp[s];
                pair(e, c1, c1, c1);
            }
        }
    } else {
        for (int k = 0; k < len; ++k) {
            float4 e = ldg4_stream(g + (int64_t)k * kTileRows);
            int s = min(max(__float_as_int(e.w), 0), max(m - 1, 0));
            int64_t j = min(max((int64_t)A.uidx[P0 + s], (int64_t)0), n - 1);
            const float4* rec = reinterpret_cast<const float4*>(RM + W * j);
            float4 c1 = __ldg(rec + 1);
            float4 c2 = DIM == 3 ? __ldg(rec + 2) : c1, c3 = DIM == 3 ? __ldg(rec + 3) : c1;
            pair(e, c1, c2, c3);
        }
    }
    if (!active) return;
    float2 v01 = acc01.value();
    float tot[3] = {v01.x, v01.y, DIM == 3 ? acc2.value() : 0.0f};
    if (OUT == OUT_RATES) {
        for (int a = 0; a < DIM; ++a) dvdt[a * n + i] = (double)(tot[a] * K.inv_rho0);
        return;
    }
    bool fx = (bi & kFixedBit) != 0;
    float* vrec = RD + 8 * i + 4;
#pragma unroll
    for (int a = 0; a < DIM; ++a) vrec[a] = fx ? 0.0f : vown[a] + K.dt * (tot[a] * K.inv_rho0);
}

// Geometry form of the momentum pass (Eq. 30), boxes without periodic axes.  Eq. 30's
// sum is taken in its two halves,
//   a_i = (1/rho0) (M_i S_i + sum_j (V0_j M_j) g_ij),   g_ij = (dW/dr / r)(r_ij) r_ij,
// with S_i = sum_j g_ij V0_j fixed by the reference configuration (computed in float64
// with the plan, k_tl_geo), so a pair needs the neighbour's position and V0_j M_j only and
// evaluates its kernel gradient from them instead of streaming a 16-byte factor.  The block
// stages, per distinct neighbour of its tile, the position relative to the cell of the
// tile's first row and V0_j M_j (mom_stage: 3D three float4 planes, 2D a float4 and a
// float2 plane); the pair slots come from the plan's slot section.  Without a shared slot
// block 8 blocks of 4 warps fit an SM (48 bytes per staged neighbour), which hides more of
// the staging's latency than a slot read from shared memory saves.
template <int DIM>
__device__ __forceinline__ void mom_stage_rec(const F8& a, const F8& b, uint32_t bref, const TLK<float>& K, float4& p0,
                                              float4& p1, float4& p2) {
    if (DIM == 3) {
        // record (ox, oy, oz, cell, M00, M10, M20, V0 | M01, M11, M21, 0, M02, M12, M22, 0)
        float x[3];
        rel_to_ref<3>(a.v, __float_as_uint(a.v[3]), bref, K, x);
        const float V = a.v[7];
        p0 = make_float4(x[0], x[1], x[2], V * b.v[6]);                     // x, y, z, VM22
        p1 = make_float4(V * a.v[4], V * a.v[5], V * b.v[0], V * b.v[1]);   // VM00, VM10, VM01, VM11
        p2 = make_float4(V * b.v[4], V * b.v[5], V * a.v[6], V * b.v[2]);   // VM02, VM12, VM20, VM21
    } else {
        // record (ox, oy, cell, V0, M00, M10, M01, M11)
        float x[2];
        rel_to_ref<2>(a.v, __float_as_uint(a.v[2]), bref, K, x);
        const float V = a.v[3];
        p0 = make_float4(x[0], x[1], V * a.v[4], V * a.v[5]);               // x, y, VM00, VM10
        p1 = make_float4(V * a.v[6], V * a.v[7], 0.0f, 0.0f);               // VM01, VM11
        p2 = p1;
    }
}

template <int DIM>
__device__ __forceinline__ void mom_stage(const float* __restrict__ RM, int64_t j, uint32_t bref,
                                          const TLK<float>& K, float4& p0, float4& p1, float4& p2) {
    constexpr int W = DIM == 3 ? 16 : 8;
    const F8 a = ldg8(RM + W * j);
    const F8 b = DIM == 3 ? ldg8(RM + W * j + 8) : a;
    mom_stage_rec<DIM>(a, b, bref, K, p0, p1, p2);
}

// The terms of one pair of the geometry form, (V0_j M_j) g_ij as rows 0-1 paired and row 2;
// FUSE adds them to (t01, t2) with one rounding per product (blocks of two pairs).
template <int DIM, bool FUSE>
__device__ __forceinline__ void mom_terms_rel(float4 p0, float4 p1, float4 p2, const float* xi, const TLK<float>& K,
                                              float2& t01, float& t2) {
    float r[DIM];
    r[0] = xi[0] - p0.x;
    r[1] = xi[1] - p0.y;
    if (DIM == 3) r[DIM - 1] = xi[DIM - 1] - p0.z;
    float d2 = r[0] * r[0];
#pragma unroll
    for (int a = 1; a < DIM; ++a) d2 = fmaf(r[a], r[a], d2);
    const float gs = gs_from_d2(d2, K);
    const float g0 = gs * r[0], g1 = gs * r[1];
    if (DIM == 2) {
        const float2 a0 = FUSE ? __ffma2_rn(make_float2(p0.z, p0.w), make_float2(g0, g0), t01)
                               : __fmul2_rn(make_float2(p0.z, p0.w), make_float2(g0, g0));
        t01 = __ffma2_rn(make_float2(p1.x, p1.y), make_float2(g1, g1), a0);
    } else {
        const float g2 = gs * r[DIM - 1];
        const float2 a0 = FUSE ? __ffma2_rn(make_float2(p1.x, p1.y), make_float2(g0, g0), t01)
                               : __fmul2_rn(make_float2(p1.x, p1.y), make_float2(g0, g0));
        t01 = __ffma2_rn(make_float2(p2.x, p2.y), make_float2(g2, g2),
                         __ffma2_rn(make_float2(p1.z, p1.w), make_float2(g1, g1), a0));
        t2 = fmaf(p0.w, g2, fmaf(p2.w, g1, FUSE ? fmaf(p2.z, g0, t2) : p2.z * g0));
    }
}

// One pair of the geometry form: accumulates (V0_j M_j) g_ij, rows 0-1 paired and row 2 alone.
template <int DIM>
__device__ __forceinline__ void mom_pair_rel(float4 p0, float4 p1, float4 p2, const float* xi, const TLK<float>& K,
                                             Kahan2& acc01, Kahan<float>& acc2) {
    float r[DIM];
    r[0] = xi[0] - p0.x;
    r[1] = xi[1] - p0.y;
    if (DIM == 3) r[DIM - 1] = xi[DIM - 1] - p0.z;
    float d2 = r[0] * r[0];
#pragma unroll
    for (int a = 1; a < DIM; ++a) d2 = fmaf(r[a], r[a], d2);
    const float gs = gs_from_d2(d2, K);
    const float g0 = gs * r[0], g1 = gs * r[1];
    if (DIM == 2) {
        acc01.add(__ffma2_rn(make_float2(p1.x, p1.y), make_float2(g1, g1),
                             __fmul2_rn(make_float2(p0.z, p0.w), make_float2(g0, g0))));
    } else {
        const float g2 = gs * r[DIM - 1];
        const float2 t01 = __ffma2_rn(make_float2(p2.x, p2.y), make_float2(g2, g2),
                                      __ffma2_rn(make_float2(p1.z, p1.w), make_float2(g1, g1),
                                                 __fmul2_rn(make_float2(p1.x, p1.y), make_float2(g0, g0))));
        acc01.add(t01);
        acc2.add(fmaf(p0.w, g2, fmaf(p2.w, g1, p2.z * g0)));
    }
}

template <int DIM, int OUT>
__global__ void __launch_bounds__(kTileRows, 8) k_tl_mom32r(const float* __restrict__ RM, float* __restrict__ RD,
                                                            const int64_t* __restrict__ row_ptr, int64_t n,
                                                            TLK<float> K, GeoArgs A, double* __restrict__ dvdt) {
    constexpr int W = DIM == 3 ? 16 : 8;
    extern __shared__ __align__(16) unsigned char tl_smem[];
    const int mc = A.mcap;
    float4* P0s = reinterpret_cast<float4*>(tl_smem);
    float4* P1s = P0s + mc;
    float4* P2s = P1s + mc;                                   // 3D
    float2* P1h = reinterpret_cast<float2*>(P0s + mc);        // 2D
    // tiles in reverse: the deformation pass walks them forwards, so each pass starts on
    // the records the previous one touched last, still in L2
    const int64_t tile = gridDim.x - 1 - blockIdx.x;
    const int64_t i0 = tile * kTileRows;
    const int64_t i = i0 + threadIdx.x;
    const bool active = i < n;
    const int64_t ii = active ? i : i0;
    const int64_t P0 = row_ptr[i0];
    const int len = active ? (int)(row_ptr[ii + 1] - row_ptr[ii]) : 0;
    const int m = A.tile_m[tile];
    // the cell code of the tile's first row, from RD (whose position quarter no pass writes)
    const uint32_t bref = __float_as_uint(RD[8 * i0 + DIM]);
    // pair slots are read from the plan's slot section (a warp reads 64 contiguous bytes per
    // position): without a shared slot block the stage fits 8 blocks per SM
    const bool staged = m <= mc;
    const float4 S = A.wsum[ii];
    // up to four neighbours per thread per round: their indices first, then their records
    // two at a time, so that few round trips to memory are in series
    int64_t jq[4];
    int pq[4];
    auto indices = [&](int q0) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int q = q0 + k * kTileRows + (int)threadIdx.x;
            // a plan out of date with the lists reads wrong but in-bounds records
            jq[k] = q < m ? min(max((int64_t)A.uidx[P0 + q], (int64_t)0), n - 1) : -1;
            pq[k] = q < m ? min((int)A.spos[P0 + q], m - 1) : 0;
        }
    };
    // launched as a programmatic dependent of the previous pass: everything above reads
    // the plan and the fixed lists only; the records the previous pass wrote are read after
    // the wait
    if (staged) indices(0);
    grid_dependency_wait();
    grid_launch_dependents();
    // the own record is requested before the staging: its latency overlaps it
    const F8 a0 = ldg8(RM + W * ii);
    const F8 a1 = DIM == 3 ? ldg8(RM + W * ii + 8) : a0;
    if (staged) {
        for (int q0 = 0; q0 < m; q0 += 4 * kTileRows) {
            if (q0 > 0) indices(q0);
#pragma unroll
            for (int k = 0; k < 4; k += 2) {
                F8 ra[2], rb[2];
#pragma unroll
                for (int t = 0; t < 2; ++t) {
                    const int64_t j = jq[k + t] < 0 ? 0 : jq[k + t];
                    ra[t] = ldg8(RM + W * j);
                    rb[t] = DIM == 3 ? ldg8(RM + W * j + 8) : ra[t];
                }
#pragma unroll
                for (int t = 0; t < 2; ++t) {
                    if (jq[k + t] < 0) continue;
                    const int q = pq[k + t];
                    float4 p0, p1, p2;
                    mom_stage_rec<DIM>(ra[t], rb[t], bref, K, p0, p1, p2);
                    P0s[q] = p0;
                    if (DIM == 3) {
                        P1s[q] = p1;
                        P2s[q] = p2;
                    } else {
                        P1h[q] = make_float2(p1.x, p1.y);
                    }
                }
            }
        }
    }
    __syncthreads();
    // M_i S_i is the sums' first term, so M_i is not kept through the loop
    float xi[3] = {0.0f, 0.0f, 0.0f};
    Kahan2 acc01;
    Kahan<float> acc2;
    acc01.init();
    acc2.init();
    uint32_t bi;
    {
        bi = __float_as_uint(a0.v[DIM]);
        rel_to_ref<DIM>(a0.v, bi, bref, K, xi);
        float2 mi01[DIM];
        float mi2[3] = {0.0f, 0.0f, 0.0f};
        own_M<DIM>(a0, a1, mi01, mi2);
        if (DIM == 2) {
            acc01.add(__ffma2_rn(mi01[1], make_float2(S.y, S.y), __fmul2_rn(mi01[0], make_float2(S.x, S.x))));
        } else {
            acc01.add(__ffma2_rn(mi01[DIM - 1], make_float2(S.z, S.z),
                                 __ffma2_rn(mi01[1], make_float2(S.y, S.y), __fmul2_rn(mi01[0], make_float2(S.x, S.x)))));
            acc2.add(fmaf(mi2[2], S.z, fmaf(mi2[1], S.y, mi2[0] * S.x)));
        }
    }
    const int mlast = max(m - 1, 0);
    const uint16_t* gsl = A.slots + A.tile_so[tile] + threadIdx.x;
    if (staged) {
        // pairs in blocks of two: each block's terms summed with one rounding per product,
        // then added to the compensated sums
        auto planes = [&](int s, float4& p0, float4& p1, float4& p2) {
            p0 = P0s[s];
            if (DIM == 3) {
                p1 = P1s[s];
                p2 = P2s[s];
            } else {
                const float2 h = P1h[s];
                p1 = make_float4(h.x, h.y, 0.0f, 0.0f);
                p2 = p1;
            }
        };
        // the next block's slots are requested before this block's pairs are evaluated
        int k = 0;
        int s0n = len > 0 ? min((int)__ldg(gsl), mlast) : 0;
        int s1n = len > 1 ? min((int)__ldg(gsl + kTileRows), mlast) : 0;
#pragma unroll 2
        for (; k + 1 < len; k += 2) {
            const int s0 = s0n, s1 = s1n;
            s0n = k + 2 < len ? min((int)__ldg(gsl + (int64_t)(k + 2) * kTileRows), mlast) : 0;
            s1n = k + 3 < len ? min((int)__ldg(gsl + (int64_t)(k + 3) * kTileRows), mlast) : 0;
            float4 a0, a1, a2, b0, b1, b2;
            planes(s0, a0, a1, a2);
            planes(s1, b0, b1, b2);
            float2 t01;
            float t2 = 0.0f;
            mom_terms_rel<DIM, false>(a0, a1, a2, xi, K, t01, t2);
            mom_terms_rel<DIM, true>(b0, b1, b2, xi, K, t01, t2);
            acc01.add(t01);
            if (DIM == 3) acc2.add(t2);
        }
        if (k < len) {
            const int s0 = s0n;
            float4 a0, a1, a2;
            planes(s0, a0, a1, a2);
            float2 t01;
            float t2 = 0.0f;
            mom_terms_rel<DIM, false>(a0, a1, a2, xi, K, t01, t2);
            acc01.add(t01);
            if (DIM == 3) acc2.add(t2);
        }
    } else {
        for (int k = 0; k < len; ++k) {
            const int s = min((int)__ldg(gsl + (int64_t)k * kTileRows), mlast);
            const int q = min((int)A.sinv[P0 + s], mlast);
            const int64_t j = min(max((int64_t)A.uidx[P0 + q], (int64_t)0), n - 1);
            float4 p0, p1, p2;
            mom_stage<DIM>(RM, j, bref, K, p0, p1, p2);
            mom_pair_rel<DIM>(p0, p1, p2, xi, K, acc01, acc2);
        }
    }
    if (!active) return;
    const float2 v01 = acc01.value();
    const float tot[3] = {v01.x, v01.y, DIM == 3 ? acc2.value() : 0.0f};
    if (OUT == OUT_RATES) {
        for (int a = 0; a < DIM; ++a) dvdt[a * n + i] = (double)(tot[a] * K.inv_rho0);
        return;
    }
    // the velocity quarter of the RD record, (vx, vy, vz, V0) in 3D and (vx, vy, 0, 0) in
    // 2D, read and written as one float4
    const bool fx = (bi & kFixedBit) != 0;
    float4* vrec = reinterpret_cast<float4*>(RD + 8 * i + 4);
    float4 vv = *vrec;
    float* vp = reinterpret_cast<float*>(&vv);
#pragma unroll
    for (int a = 0; a < DIM; ++a) vp[a] = fx ? 0.0f : vp[a] + K.dt * (tot[a] * K.inv_rho0);
    *vrec = vv;
}

// BULK: thread 0 copies the tile's whole entry block into shared memory with one
// TMA bulk copy (completion on an mbarrier, bounded wait) while the block stages
// the neighbours, so each block has its entire entry stream in flight at once;
// tiles with more than A.ecap entries stream them from global memory as without.
// GEOM: the pair geometry from the staged records (both halves of RD: position code and
// velocity) and the sliced slot section, instead of the 16-byte entries: 2 bytes of the
// plan per pair instead of 16, for about 30 more instructions per pair.
// HX: the new H and u are also written to Hx, ux (mapped host memory of a caller that keeps
// the state on the host), so that the write-back overlaps the pass.
template <int DIM, int OUT, bool BULK, bool GEOM = false, bool PER = false, bool HX = false>
__global__ void __launch_bounds__(kTileRows, BULK ? 3 : (GEOM ? 8 : 6)) k_tl_defo32g(
    const float* __restrict__ RD, float* __restrict__ RM, const int64_t* __restrict__ row_ptr, int64_t n,
    TLK<float> K, GeoArgs A, const float* __restrict__ B0, float* __restrict__ H, float* __restrict__ u,
    double* __restrict__ dFdt, int* __restrict__ flags, float* __restrict__ Hx, float* __restrict__ ux) {
    constexpr int NS = DIM == 2 ? 3 : 6;
    extern __shared__ __align__(16) unsigned char tl_smem[];
    float4* sp = reinterpret_cast<float4*>(tl_smem);
    const int64_t tile = blockIdx.x;
    const int64_t i0 = tile * kTileRows;
    const int64_t i = i0 + threadIdx.x;
    const bool active = i < n;
    const int64_t ii = active ? i : i0;
    float4* eb = sp + A.mcap;
    uint64_t* bar = reinterpret_cast<uint64_t*>(eb + A.ecap);
    const int te = BULK ? A.tile_e[tile] : 0;
    const bool bulk = BULK && te > 0 && te <= A.ecap;
    // A.test_polls > 0 (failure-detection test): no copy is issued, so the bounded wait
    // below runs out on a phase nothing completes and the block leaves with nothing in flight
    const bool test_wait = BULK && A.test_polls > 0;
    if (BULK && threadIdx.x == 0) {
        mbar_init(bar, 1);
        mbar_fence_init();
        if (bulk && !test_wait) {
            mbar_arrive_expect_tx(bar, (uint32_t)te * 16u);
            tma_load_1d(eb, A.geo + A.tile_so[tile], (uint32_t)te * 16u, bar);
        }
    }
    const int64_t P0 = row_ptr[i0];
    const int len = active ? (int)(row_ptr[ii + 1] - row_ptr[ii]) : 0;
    const int m = A.tile_m[tile];
    const float4* g = A.geo + A.tile_so[tile] + threadIdx.x;
    float b0[NS], hold[DIM * DIM], uold[DIM];
    // the epilogue's own-row reads: issued here, their latency hidden by the loop, or (the
    // geometry form) after it, to keep 18 registers free for more resident warps
    auto own_row = [&]() {
#pragma unroll
        for (int s = 0; s < NS; ++s) b0[s] = B0[s * n + ii];
#pragma unroll
        for (int k = 0; k < DIM * DIM; ++k) hold[k] = OUT == OUT_RATES ? 0.0f : H[k * n + ii];
#pragma unroll
        for (int a = 0; a < DIM; ++a) uold[a] = OUT == OUT_RATES ? 0.0f : u[a * n + ii];
    };
    // GEOM without periodic axes: positions staged relative to the cell of the tile's
    // first row (decoded once per neighbour, not per pair)
    constexpr bool REL = GEOM && !PER;
    const uint32_t bref = REL ? __float_as_uint(RD[8 * i0 + DIM]) : 0u;
    // REL: the tile's slot block (its entries' 2-byte slots, 256 bytes per position, one
    // contiguous range of the plan) copied into shared memory after the two staged planes by
    // one TMA bulk copy, issued first (plan data: before the dependency wait) and completed
    // on an mbarrier (bounded wait), when the plan's longest row allows (A.ecap positions).
    // A.test_polls > 0 (failure-detection test): no copy, and the wait runs out.
    uint16_t* ssl = reinterpret_cast<uint16_t*>(sp + 2 * A.mcap);
    uint64_t* sbar = reinterpret_cast<uint64_t*>(reinterpret_cast<unsigned char*>(ssl) + (size_t)A.ecap * kTileRows * 2);
    const int width = REL ? A.tile_e[tile] / kTileRows : 0;
    const bool sslot = REL && width <= A.ecap;
    const bool slot_test = sslot && A.test_polls > 0;
    if (sslot && threadIdx.x == 0) {
        mbar_init(sbar, 1);
        mbar_fence_init();
        if (!slot_test) {
            const uint32_t bytes = (uint32_t)width * kTileRows * 2u;
            mbar_arrive_expect_tx(sbar, bytes);
            tma_load_1d(ssl, A.slots + A.tile_so[tile], bytes, sbar);
        }
    }
    // up to four neighbours per thread per round: their indices first, then their records
    // two at a time, so that few round trips to memory are in series
    int64_t jq[4];
    int pq[4];
    auto indices = [&](int q0) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int q = q0 + k * kTileRows + (int)threadIdx.x;
            jq[k] = q < m ? min(max((int64_t)A.uidx[P0 + q], (int64_t)0), n - 1) : -1;
            pq[k] = q < m ? min((int)A.spos[P0 + q], m - 1) : 0;
        }
    };
    bool staged = REL ? m <= A.mcap : false;
    // launched as a programmatic dependent of the previous pass: everything above reads
    // the plan, the fixed lists and RD's position quarter (which no pass writes); RD's
    // velocities, H and u are read after the wait
    if (REL && staged) indices(0);
    grid_dependency_wait();
    grid_launch_dependents();
    F8 me = ldg8(RD + 8 * ii);
    if (!GEOM) own_row();
    if (REL) {
        if (staged) {
            for (int q0 = 0; q0 < m; q0 += 4 * kTileRows) {
                if (q0 > 0) indices(q0);
#pragma unroll
                for (int k = 0; k < 4; k += 2) {
                    F8 rr[2];
#pragma unroll
                    for (int t = 0; t < 2; ++t) rr[t] = ldg8(RD + 8 * (jq[k + t] < 0 ? 0 : jq[k + t]));
#pragma unroll
                    for (int t = 0; t < 2; ++t) {
                        if (jq[k + t] < 0) continue;
                        const int q = pq[k + t];
                        float x[3] = {0.0f, 0.0f, 0.0f};
                        rel_to_ref<DIM>(rr[t].v, __float_as_uint(rr[t].v[DIM]), bref, K, x);
                        sp[q] = make_float4(x[0], x[1], x[2], DIM == 3 ? rr[t].v[7] : rr[t].v[3]);
                        sp[A.mcap + q] = hi4(rr[t]);
                    }
                }
            }
        }
        __syncthreads();
        if (sslot) {
            const bool late = !mbar_wait_bounded(sbar, 0, slot_test ? A.test_polls : kWaitPolls);
            if (__syncthreads_or(late)) {      // block-uniform: the copy never completed
                if (threadIdx.x == 0) atomicExch(&flags[FLAG_TIMEOUT], 1);
                if (!slot_test) mbar_wait_bounded(sbar, 0, kWaitPolls);    // a copy issued is waited for
                return;
            }
        }
    } else {
        staged = GEOM ? stage_neighbours<2, 8, 0>(RD, n, P0, m, A, sp, A.spos)
                      : stage_neighbours<1, 8>(RD, n, P0, m, A, sp);
    }
    if (bulk) {
        const bool late = !mbar_wait_bounded(bar, 0, test_wait ? A.test_polls : kWaitPolls);
        if (__syncthreads_or(late)) {      // block-uniform: the copy never completed
            if (threadIdx.x == 0) atomicExch(&flags[FLAG_TIMEOUT], 1);
            if (!test_wait) mbar_wait_bounded(bar, 0, kWaitPolls);    // a copy issued is waited for
            return;
        }
    }
    const uint32_t bi = __float_as_uint(me.v[DIM]);
    const float2 nv01 = make_float2(-me.v[4], -me.v[5]);
    const float nv2 = -me.v[6];
    Kahan2 c01[DIM];
    Kahan2 r2;
    Kahan<float> l22;
#pragma unroll
    for (int c = 0; c < DIM; ++c) c01[c].init();
    r2.init();
    l22.init();
    auto pair = [&](float4 e, float4 vj) {
        float2 dv01 = __fadd2_rn(make_float2(vj.x, vj.y), nv01);
        c01[0].add(__fmul2_rn(dv01, make_float2(e.x, e.x)));
        c01[1].add(__fmul2_rn(dv01, make_float2(e.y, e.y)));
        if (DIM == 3) {
            float dv2 = vj.z + nv2;
            c01[DIM - 1].add(__fmul2_rn(dv01, make_float2(e.z, e.z)));
            r2.add(__fmul2_rn(make_float2(dv2, dv2), make_float2(e.x, e.y)));
            l22.add(dv2 * e.z);
        }
    };
    if (REL && staged) {
        float xi[3] = {0.0f, 0.0f, 0.0f};
        rel_to_ref<DIM>(me.v, bi, bref, K, xi);
        if (sslot) {
            // pairs in blocks of four: each block's products summed with one rounding per
            // term, then added to the compensated sums
            const uint16_t* sl = ssl + threadIdx.x;
            const int mlast = max(m - 1, 0);
            int k = 0;
            for (; k + 3 < len; k += 4) {
                const int s0 = min((int)sl[k * kTileRows], mlast), s1 = min((int)sl[(k + 1) * kTileRows], mlast);
                const int s2 = min((int)sl[(k + 2) * kTileRows], mlast), s3 = min((int)sl[(k + 3) * kTileRows], mlast);
                DefoTerms t;
                defo_terms_rel<DIM, false>(sp[s0], sp[A.mcap + s0], xi, nv01, nv2, K, t);
                defo_terms_rel<DIM, true>(sp[s1], sp[A.mcap + s1], xi, nv01, nv2, K, t);
                defo_terms_rel<DIM, true>(sp[s2], sp[A.mcap + s2], xi, nv01, nv2, K, t);
                defo_terms_rel<DIM, true>(sp[s3], sp[A.mcap + s3], xi, nv01, nv2, K, t);
                defo_add_terms<DIM>(t, c01, r2, l22);
            }
            if (k < len) {
                DefoTerms t;
                int s0 = min((int)sl[k * kTileRows], mlast);
                defo_terms_rel<DIM, false>(sp[s0], sp[A.mcap + s0], xi, nv01, nv2, K, t);
                for (++k; k < len; ++k) {
                    s0 = min((int)sl[k * kTileRows], mlast);
                    defo_terms_rel<DIM, true>(sp[s0], sp[A.mcap + s0], xi, nv01, nv2, K, t);
                }
                defo_add_terms<DIM>(t, c01, r2, l22);
            }
        } else {
            const uint16_t* sl = A.slots + A.tile_so[tile] + threadIdx.x;
#pragma unroll 4
            for (int k = 0; k < len; ++k) {
                int s = min((int)__ldg(sl + (int64_t)k * kTileRows), max(m - 1, 0));
                defo_pair_rel<DIM>(sp[s], sp[A.mcap + s], xi, nv01, nv2, K, c01, r2, l22);
            }
        }
    } else if (GEOM) {
        float oi[DIM];
#pragma unroll
        for (int a = 0; a < DIM; ++a) oi[a] = me.v[a];
        const uint16_t* sl = A.slots + A.tile_so[tile] + threadIdx.x;
        if (staged) {
#pragma unroll 4
            for (int k = 0; k < len; ++k) {
                int s = min((int)__ldg(sl + (int64_t)k * kTileRows), max(m - 1, 0));
                defo_pair<DIM, PER>(sp[s], sp[A.mcap + s], oi, bi, nv01, nv2, K, c01, r2, l22);
            }
        } else {
            for (int k = 0; k < len; ++k) {
                int s = min((int)__ldg(sl + (int64_t)k * kTileRows), max(m - 1, 0));
                const int q = min((int)A.sinv[P0 + s], max(m - 1, 0));
                int64_t j = min(max((int64_t)A.uidx[P0 + q], (int64_t)0), n - 1);
                F8 rj = ldg8(RD + 8 * j);
                defo_pair<DIM, PER>(lo4(rj), hi4(rj), oi, bi, nv01, nv2, K, c01, r2, l22);
            }
        }
    } else if (bulk && staged) {
        const float4* gs = eb + threadIdx.x;
#pragma unroll 4
        for (int k = 0; k < len; ++k) {
            float4 e = gs[k * kTileRows];
            int s = min(max(__float_as_int(e.w), 0), max(m - 1, 0));
            pair(e, sp[s]);
        }
    } else if (staged) {
#pragma unroll 4
        for (int k = 0; k < len; ++k) {
            float4 e = ldg4_stream(g + (int64_t)k * kTileRows);
            int s = min(max(__float_as_int(e.w), 0), max(m - 1, 0));
            pair(e, sp[s]);
        }
    } else {
        for (int k = 0; k < len; ++k) {
            float4 e = bulk ? eb[threadIdx.x + k * kTileRows] : ldg4_stream(g + (int64_t)k * kTileRows);
            int s = min(max(__float_as_int(e.w), 0), max(m - 1, 0));
            int64_t j = min(max((int64_t)A.uidx[P0 + s], (int64_t)0), n - 1);
            pair(e, __ldg(reinterpret_cast<const float4*>(RD + 8 * j) + 1));
        }
    }
    if (!active) return;
    float Lt[DIM * DIM];
#pragma unroll
    for (int c = 0; c < DIM; ++c) {
        float2 v = c01[c].value();
        Lt[0 * DIM + c] = v.x;
        Lt[1 * DIM + c] = v.y;
    }
    if (DIM == 3) {
        float2 v = r2.value();
        Lt[2 * DIM + 0] = v.x;
        Lt[2 * DIM + 1] = v.y;
        Lt[2 * DIM + 2] = l22.value();
    }
    float vi[3] = {me.v[4], me.v[5], me.v[6]};
    // the own record again, with the epilogue's other own-row reads (keeping the first
    // read live through the loop costs registers there)
    const F8 own = ldg8(RD + 8 * i);
    if (GEOM) own_row();
    defo_finish<DIM, OUT>(Lt, b0, (bi & kFixedBit) != 0, vi, i, n, K, RM, H, u, dFdt, hold, uold, &own,
                          HX ? Hx : nullptr, HX ? ux : nullptr);
}

// ---------------------------------------------------------------- pack / unpack
template <int DIM>
__global__ void k_tl_pack(const double* __restrict__ r0, const double* __restrict__ V0,
                          const double* __restrict__ B0, const uint8_t* __restrict__ fixed,
                          const double* __restrict__ x, const double* __restrict__ v,
                          const double* __restrict__ H, int64_t n, RelGrid g, float* __restrict__ RD,
                          float* __restrict__ RM, float* __restrict__ H32, float* __restrict__ u32,
                          float* __restrict__ B32) {
    constexpr int NS = DIM == 2 ? 3 : 6;
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float o[3] = {0, 0, 0};
    double xr[3] = {0, 0, 0};
    for (int a = 0; a < DIM; ++a) xr[a] = r0[a * n + i];
    uint32_t bits = rel_encode<DIM>(xr, g, o);
    if (fixed && fixed[i]) bits |= kFixedBit;
    float V = (float)V0[i];
    float vv[3] = {0, 0, 0};
    for (int a = 0; a < DIM; ++a) vv[a] = (float)v[a * n + i];
    float* d = RD + 8 * i;
    float* m = RM + (DIM == 3 ? 16 : 8) * i;
    if (DIM == 3) {
        d[0] = o[0]; d[1] = o[1]; d[2] = o[2]; d[3] = __uint_as_float(bits);
        d[4] = vv[0]; d[5] = vv[1]; d[6] = vv[2]; d[7] = V;
        for (int k = 0; k < 16; ++k) m[k] = 0.0f;
        m[0] = o[0]; m[1] = o[1]; m[2] = o[2]; m[3] = __uint_as_float(bits); m[7] = V;
    } else {
        d[0] = o[0]; d[1] = o[1]; d[2] = __uint_as_float(bits); d[3] = V;
        d[4] = vv[0]; d[5] = vv[1]; d[6] = 0.0f; d[7] = 0.0f;
        for (int k = 0; k < 8; ++k) m[k] = 0.0f;
        m[0] = o[0]; m[1] = o[1]; m[2] = __uint_as_float(bits); m[3] = V;
    }
    for (int k = 0; k < DIM * DIM; ++k) H32[k * n + i] = (float)H[k * n + i];
    for (int a = 0; a < DIM; ++a) u32[a * n + i] = (float)(x[a * n + i] - r0[a * n + i]);
    for (int s = 0; s < NS; ++s) B32[s * n + i] = (float)B0[s * n + i];
}

template <int DIM>
__global__ void k_tl_unpack(const double* __restrict__ r0, const float* __restrict__ RD,
                            const float* __restrict__ H32, const float* __restrict__ u32, int64_t n,
                            double* __restrict__ x, double* __restrict__ v, double* __restrict__ H) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int a = 0; a < DIM; ++a) {
        v[a * n + i] = RD[8 * i + 4 + a];
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

int check_tl(const sph_tlsph_params* p, const sph_tlsph_state* st) {
    if (!p || !st) return SPH_ERR_ARG;
    int s = sph_check_domain(&p->dom);
    if (s) return s;
    if (p->precision != SPH_FP64 && p->precision != SPH_FP32_KAHAN) return SPH_ERR_ARG;
    if (p->law != SPH_SVK && p->law != SPH_NEO_HOOKEAN) return SPH_ERR_ARG;
    if (!(p->rho0 > 0.0)) return SPH_ERR_ARG;
    if (p->dom.n > 0 && (!st->row_ptr || !st->col || !st->r0 || !st->V0 || !st->B0)) return SPH_ERR_ARG;
    if (p->precision == SPH_FP32_KAHAN) {
        // the cell-relative minimum image needs len >= 2 kappa h + 2 S on periodic axes
        if (!rel_grid_periodic_ok(make_rel_grid(p->dom), p->dom.dim, p->dom.kappa * p->dom.h)) return SPH_ERR_ARG;
    }
    return SPH_OK;
}

// --------------------------- persistent, double-buffered form of the planned passes
// One block per SM walks the tiles b, b + G, b + 2G, ... (G blocks).  While it
// computes tile t, the TMA unit copies tile t+G's sliced pair entries into the
// other entry buffer (completion on an mbarrier), per-thread asynchronous copies
// stage t+G's neighbour chunks (from the list copied one tile earlier) and t+2G's
// neighbour list, and the row's own data for t+G is loaded into registers.  Used
// when both entry buffers fit in shared memory.
struct PipeArgs {
    int64_t ntiles;
    int gw;      // entries per buffer: kTileRows * longest row
    int mcap;    // neighbours staged per tile
    int ucap;    // ints per list buffer
};

struct TileHdr {
    int m, ne;
    int64_t P0, so;
};

__device__ __forceinline__ TileHdr tile_hdr(const GeoArgs& A, const int64_t* __restrict__ row_ptr, int64_t t,
                                            int64_t ntiles) {
    TileHdr h{0, 0, 0, 0};
    if (t < ntiles) {
        h.m = A.tile_m[t];
        h.so = A.tile_so[t];
        h.ne = (int)(A.tile_so[t + 1] - h.so);
        h.P0 = row_ptr[t * kTileRows];
    }
    return h;
}

template <int NPL>
struct PipeSmem {
    uint64_t* bar;
    float4* gbuf;
    float4* rbuf;
    int32_t* ubuf;
    __device__ PipeSmem(unsigned char* base, const PipeArgs& P) {
        bar = reinterpret_cast<uint64_t*>(base);
        gbuf = reinterpret_cast<float4*>(base + 16);
        rbuf = gbuf + 2 * (size_t)P.gw;
        ubuf = reinterpret_cast<int32_t*>(rbuf + 2 * (size_t)NPL * P.mcap);
    }
};

static inline size_t pipe_smem_bytes(const PipeArgs& P, int npl) {
    return 16 + 2 * (size_t)P.gw * 16 + 2 * (size_t)npl * P.mcap * 16 + 3 * (size_t)P.ucap * 4;
}

// Copy the neighbour list of tile t (when it will be staged) into ub.
__device__ __forceinline__ void issue_list(const GeoArgs& A, const PipeArgs& P, int64_t t, const TileHdr& h,
                                           int32_t* ub) {
    if (t < P.ntiles && h.m <= P.mcap)
        for (int s = threadIdx.x; s < h.m; s += blockDim.x) cp_async4(ub + s, A.uidx + h.P0 + s);
}

// Start tile t's entry copy (thread 0, on bar) and its neighbour chunks 1..NPL.
template <int NPL, int RECF>
__device__ __forceinline__ void issue_tile(const GeoArgs& A, const PipeArgs& P, const float* __restrict__ R,
                                           int64_t n, int64_t t, const TileHdr& h, int b, const PipeSmem<NPL>& S,
                                           const int32_t* ub) {
    if (t >= P.ntiles) return;
    if (threadIdx.x == 0) {
        uint32_t bytes = (uint32_t)h.ne * 16u;
        mbar_arrive_expect_tx(&S.bar[b], bytes);
        if (bytes) tma_load_1d(S.gbuf + (size_t)b * P.gw, A.geo + h.so, bytes, &S.bar[b]);
    }
    if (h.m <= P.mcap) {
        float4* rb = S.rbuf + (size_t)b * NPL * P.mcap;
        for (int s = threadIdx.x; s < h.m; s += blockDim.x) {
            int64_t j = min(max((int64_t)ub[s], (int64_t)0), n - 1);
            const float4* src = reinterpret_cast<const float4*>(R + RECF * j) + 1;
#pragma unroll
            for (int c = 0; c < NPL; ++c) cp_async16(rb + (size_t)c * P.mcap + s, src + c);
        }
    }
}

struct OwnMom {
    int len;
    uint32_t bits;
    float2 mi01[3];
    float mi2[3];
    float v[3];
};

template <int DIM, int OUT>
__device__ __forceinline__ OwnMom own_mom(const float* __restrict__ RM, const float* __restrict__ RD,
                                          const int64_t* __restrict__ row_ptr, int64_t i, int64_t n) {
    constexpr int W = DIM == 3 ? 16 : 8;
    OwnMom o;
    bool active = i < n;
    int64_t ii = active ? i : n - 1;
    o.len = active ? (int)(row_ptr[ii + 1] - row_ptr[ii]) : 0;
    F8 a0 = ldg8(RM + W * ii);
    F8 a1 = DIM == 3 ? ldg8(RM + W * ii + 8) : a0;
    o.bits = __float_as_uint(a0.v[DIM]);
    o.mi2[0] = o.mi2[1] = o.mi2[2] = 0.0f;
    own_M<DIM>(a0, a1, o.mi01, o.mi2);
#pragma unroll
    for (int a = 0; a < 3; ++a) o.v[a] = (OUT != OUT_RATES && a < DIM) ? RD[8 * ii + 4 + a] : 0.0f;
    return o;
}

template <int DIM, int OUT>
__global__ void __launch_bounds__(kTileRows, 1) k_tl_mom32p(const float* __restrict__ RM, float* __restrict__ RD,
                                                            const int64_t* __restrict__ row_ptr, int64_t n,
                                                            TLK<float> K, GeoArgs A, PipeArgs P,
                                                            double* __restrict__ dvdt, int* __restrict__ flags) {
    constexpr int W = DIM == 3 ? 16 : 8;
    constexpr int NPL = DIM == 3 ? 3 : 1;
    extern __shared__ __align__(16) unsigned char tl_smem[];
    PipeSmem<NPL> S(tl_smem, P);
    const int64_t G = gridDim.x, t0 = blockIdx.x;
    if (t0 >= P.ntiles) return;
    if (threadIdx.x == 0) {
        mbar_init(&S.bar[0], 1);
        mbar_init(&S.bar[1], 1);
        mbar_fence_init();
    }
    __syncthreads();
    TileHdr h0 = tile_hdr(A, row_ptr, t0, P.ntiles), h1 = tile_hdr(A, row_ptr, t0 + G, P.ntiles);
    TileHdr h2 = tile_hdr(A, row_ptr, t0 + 2 * G, P.ntiles);
    issue_list(A, P, t0, h0, S.ubuf);
    issue_list(A, P, t0 + G, h1, S.ubuf + P.ucap);
    cp_async_commit();
    cp_async_wait_all();
    __syncthreads();
    issue_tile<NPL, W>(A, P, RM, n, t0, h0, 0, S, S.ubuf);
    cp_async_commit();
    OwnMom own = own_mom<DIM, OUT>(RM, RD, row_ptr, t0 * kTileRows + threadIdx.x, n);
    bool ok = true;
    for (int64_t it = 0;; ++it) {
        const int64_t t = t0 + it * G;
        if (t >= P.ntiles) break;
        const int cur = (int)(it & 1);
        TileHdr h3 = tile_hdr(A, row_ptr, t + 3 * G, P.ntiles);
        cp_async_wait_all();
        const bool late = !mbar_wait_bounded(&S.bar[cur], (uint32_t)((it >> 1) & 1), kWaitPolls);
        // block-uniform decision: every thread leaves the loop together
        if (__syncthreads_or(late)) {
            ok = false;
            if (threadIdx.x == 0) atomicExch(&flags[FLAG_TIMEOUT], 1);
            break;
        }
        issue_tile<NPL, W>(A, P, RM, n, t + G, h1, cur ^ 1, S, S.ubuf + ((it + 1) % 3) * P.ucap);
        issue_list(A, P, t + 2 * G, h2, S.ubuf + ((it + 2) % 3) * P.ucap);
        cp_async_commit();
        OwnMom nxt = own_mom<DIM, OUT>(RM, RD, row_ptr, (t + G) * kTileRows + threadIdx.x, n);
        // tile t
        const int64_t i = t * kTileRows + threadIdx.x;
        const float4* gb = S.gbuf + (size_t)cur * P.gw + threadIdx.x;
        const float4* rb = S.rbuf + (size_t)cur * NPL * P.mcap;
        const bool staged = h0.m <= P.mcap;
        const int smax = max(h0.m - 1, 0);
        Kahan2 acc01;
        Kahan<float> acc2;
        acc01.init();
        acc2.init();
#pragma unroll 4
        for (int k = 0; k < own.len; ++k) {
            float4 e = gb[(size_t)k * kTileRows];
            int s = min(max(__float_as_int(e.w), 0), smax);
            float4 c1, c2, c3;
            if (staged) {
                c1 = rb[s];
                c2 = DIM == 3 ? rb[P.mcap + s] : c1;
                c3 = DIM == 3 ? rb[2 * P.mcap + s] : c1;
            } else {
                int64_t j = min(max((int64_t)A.uidx[h0.P0 + s], (int64_t)0), n - 1);
                const float4* rec = reinterpret_cast<const float4*>(RM + W * j);
                c1 = __ldg(rec + 1);
                c2 = DIM == 3 ? __ldg(rec + 2) : c1;
                c3 = DIM == 3 ? __ldg(rec + 3) : c1;
            }
            if (DIM == 2) {
                float2 s0 = __fadd2_rn(own.mi01[0], make_float2(c1.x, c1.y));
                float2 s1 = __fadd2_rn(own.mi01[1], make_float2(c1.z, c1.w));
                acc01.add(__ffma2_rn(s1, make_float2(e.y, e.y), __fmul2_rn(s0, make_float2(e.x, e.x))));
            } else {
                float2 s0 = __fadd2_rn(own.mi01[0], make_float2(c1.x, c1.y));
                float2 s1 = __fadd2_rn(own.mi01[1], make_float2(c2.x, c2.y));
                float2 s2 = __fadd2_rn(own.mi01[DIM - 1], make_float2(c3.x, c3.y));
                float2 t01 = __ffma2_rn(s2, make_float2(e.z, e.z),
                                        __ffma2_rn(s1, make_float2(e.y, e.y),
                                                   __fmul2_rn(s0, make_float2(e.x, e.x))));
                float t2 = fmaf(own.mi2[2] + c3.z, e.z, fmaf(own.mi2[1] + c2.z, e.y, (own.mi2[0] + c1.z) * e.x));
                acc01.add(t01);
                acc2.add(t2);
            }
        }
        if (i < n) {
            float2 v01 = acc01.value();
            float tot[3] = {v01.x, v01.y, DIM == 3 ? acc2.value() : 0.0f};
            if (OUT == OUT_RATES) {
                for (int a = 0; a < DIM; ++a) dvdt[a * n + i] = (double)(tot[a] * K.inv_rho0);
            } else {
                bool fx = (own.bits & kFixedBit) != 0;
                float* vrec = RD + 8 * i + 4;
#pragma unroll
                for (int a = 0; a < DIM; ++a) vrec[a] = fx ? 0.0f : own.v[a] + K.dt * (tot[a] * K.inv_rho0);
            }
        }
        __syncthreads();
        own = nxt;
        h0 = h1;
        h1 = h2;
        h2 = h3;
    }
    if (!ok) {
        // let the copies in flight land before the block's shared memory is released
        cp_async_wait_all();
        mbar_wait_bounded(&S.bar[0], 0, kWaitPolls);
        mbar_wait_bounded(&S.bar[1], 0, kWaitPolls);
    }
}

template <int DIM>
struct OwnDefo {
    int len;
    uint32_t bits;
    float v[3];
    float b0[DIM == 2 ? 3 : 6];
    float h[DIM * DIM];
    float u[DIM];
};

template <int DIM, int OUT>
__device__ __forceinline__ OwnDefo<DIM> own_defo(const float* __restrict__ RD, const int64_t* __restrict__ row_ptr,
                                                 const float* __restrict__ B0, const float* __restrict__ H,
                                                 const float* __restrict__ u, int64_t i, int64_t n) {
    constexpr int NS = DIM == 2 ? 3 : 6;
    OwnDefo<DIM> o;
    bool active = i < n;
    int64_t ii = active ? i : n - 1;
    o.len = active ? (int)(row_ptr[ii + 1] - row_ptr[ii]) : 0;
    F8 me = ldg8(RD + 8 * ii);
    o.bits = __float_as_uint(me.v[DIM]);
    o.v[0] = me.v[4]; o.v[1] = me.v[5]; o.v[2] = me.v[6];
#pragma unroll
    for (int s = 0; s < NS; ++s) o.b0[s] = B0[s * n + ii];
#pragma unroll
    for (int k = 0; k < DIM * DIM; ++k) o.h[k] = OUT == OUT_RATES ? 0.0f : H[k * n + ii];
#pragma unroll
    for (int a = 0; a < DIM; ++a) o.u[a] = OUT == OUT_RATES ? 0.0f : u[a * n + ii];
    return o;
}

template <int DIM, int OUT>
__global__ void __launch_bounds__(kTileRows, 1) k_tl_defo32p(const float* __restrict__ RD, float* __restrict__ RM,
                                                             const int64_t* __restrict__ row_ptr, int64_t n,
                                                             TLK<float> K, GeoArgs A, PipeArgs P,
                                                             const float* __restrict__ B0, float* __restrict__ H,
                                                             float* __restrict__ u, double* __restrict__ dFdt,
                                                             int* __restrict__ flags) {
    extern __shared__ __align__(16) unsigned char tl_smem[];
    PipeSmem<1> S(tl_smem, P);
    const int64_t G = gridDim.x, t0 = blockIdx.x;
    if (t0 >= P.ntiles) return;
    if (threadIdx.x == 0) {
        mbar_init(&S.bar[0], 1);
        mbar_init(&S.bar[1], 1);
        mbar_fence_init();
    }
    __syncthreads();
    TileHdr h0 = tile_hdr(A, row_ptr, t0, P.ntiles), h1 = tile_hdr(A, row_ptr, t0 + G, P.ntiles);
    TileHdr h2 = tile_hdr(A, row_ptr, t0 + 2 * G, P.ntiles);
    issue_list(A, P, t0, h0, S.ubuf);
    issue_list(A, P, t0 + G, h1, S.ubuf + P.ucap);
    cp_async_commit();
    cp_async_wait_all();
    __syncthreads();
    issue_tile<1, 8>(A, P, RD, n, t0, h0, 0, S, S.ubuf);
    cp_async_commit();
    OwnDefo<DIM> own = own_defo<DIM, OUT>(RD, row_ptr, B0, H, u, t0 * kTileRows + threadIdx.x, n);
    bool ok = true;
    for (int64_t it = 0;; ++it) {
        const int64_t t = t0 + it * G;
        if (t >= P.ntiles) break;
        const int cur = (int)(it & 1);
        TileHdr h3 = tile_hdr(A, row_ptr, t + 3 * G, P.ntiles);
        cp_async_wait_all();
        const bool late = !mbar_wait_bounded(&S.bar[cur], (uint32_t)((it >> 1) & 1), kWaitPolls);
        // block-uniform decision: every thread leaves the loop together
        if (__syncthreads_or(late)) {
            ok = false;
            if (threadIdx.x == 0) atomicExch(&flags[FLAG_TIMEOUT], 1);
            break;
        }
        issue_tile<1, 8>(A, P, RD, n, t + G, h1, cur ^ 1, S, S.ubuf + ((it + 1) % 3) * P.ucap);
        issue_list(A, P, t + 2 * G, h2, S.ubuf + ((it + 2) % 3) * P.ucap);
        cp_async_commit();
        OwnDefo<DIM> nxt = own_defo<DIM, OUT>(RD, row_ptr, B0, H, u, (t + G) * kTileRows + threadIdx.x, n);
        const int64_t i = t * kTileRows + threadIdx.x;
        const float4* gb = S.gbuf + (size_t)cur * P.gw + threadIdx.x;
        const float4* rb = S.rbuf + (size_t)cur * P.mcap;
        const bool staged = h0.m <= P.mcap;
        const int smax = max(h0.m - 1, 0);
        const float2 nv01 = make_float2(-own.v[0], -own.v[1]);
        const float nv2 = -own.v[2];
        Kahan2 c01[DIM];
        Kahan2 r2;
        Kahan<float> l22;
#pragma unroll
        for (int c = 0; c < DIM; ++c) c01[c].init();
        r2.init();
        l22.init();
#pragma unroll 4
        for (int k = 0; k < own.len; ++k) {
            float4 e = gb[(size_t)k * kTileRows];
            int s = min(max(__float_as_int(e.w), 0), smax);
            float4 vj;
            if (staged) {
                vj = rb[s];
            } else {
                int64_t j = min(max((int64_t)A.uidx[h0.P0 + s], (int64_t)0), n - 1);
                vj = __ldg(reinterpret_cast<const float4*>(RD + 8 * j) + 1);
            }
            float2 dv01 = __fadd2_rn(make_float2(vj.x, vj.y), nv01);
            c01[0].add(__fmul2_rn(dv01, make_float2(e.x, e.x)));
            c01[1].add(__fmul2_rn(dv01, make_float2(e.y, e.y)));
            if (DIM == 3) {
                float dv2 = vj.z + nv2;
                c01[DIM - 1].add(__fmul2_rn(dv01, make_float2(e.z, e.z)));
                r2.add(__fmul2_rn(make_float2(dv2, dv2), make_float2(e.x, e.y)));
                l22.add(dv2 * e.z);
            }
        }
        if (i < n) {
            float Lt[DIM * DIM];
#pragma unroll
            for (int c = 0; c < DIM; ++c) {
                float2 v = c01[c].value();
                Lt[0 * DIM + c] = v.x;
                Lt[1 * DIM + c] = v.y;
            }
            if (DIM == 3) {
                float2 v = r2.value();
                Lt[2 * DIM + 0] = v.x;
                Lt[2 * DIM + 1] = v.y;
                Lt[2 * DIM + 2] = l22.value();
            }
            defo_finish<DIM, OUT>(Lt, own.b0, (own.bits & kFixedBit) != 0, own.v, i, n, K, RM, H, u, dFdt, own.h,
                                  own.u);
        }
        __syncthreads();
        own = nxt;
        h0 = h1;
        h1 = h2;
        h2 = h3;
    }
    if (!ok) {
        cp_async_wait_all();
        mbar_wait_bounded(&S.bar[0], 0, kWaitPolls);
        mbar_wait_bounded(&S.bar[1], 0, kWaitPolls);
    }
}

// The state's tile plan as launch arguments (tile_m == nullptr: no plan).
struct TlPlan {
    GeoArgs mom, defo, momr;
    PipeArgs pmom, pdefo;
    size_t mom_bytes, defo_bytes, pmom_bytes, pdefo_bytes, momr_bytes;
    bool on, pipe_mom, pipe_defo, bulk_defo, geom_defo, geom_mom;
    int grid;
};

TlPlan tl_plan(const sph_ctx* ctx, const sph_tlsph_state* st, int64_t n, int dim) {
    TlPlan t;
    t.on = st->plan && st->plan_nnz > 0 && st->plan_maxm > 0;
    t.mom = GeoArgs{nullptr, nullptr, nullptr, nullptr, 0};
    t.defo = t.mom;
    t.momr = t.mom;
    t.mom_bytes = t.defo_bytes = t.pmom_bytes = t.pdefo_bytes = t.momr_bytes = 0;
    t.pipe_mom = t.pipe_defo = t.bulk_defo = t.geom_defo = t.geom_mom = false;
    t.grid = 0;
    if (!t.on) return t;
    TilePlan tp = tile_plan_view(st->plan, n, st->plan_nnz);
    int npl = dim == 3 ? 3 : 1;
    int mm = stage_mcap(st->plan_maxm, npl, ctx->stage_cap), md = stage_mcap(st->plan_maxm, 1, ctx->stage_cap);
    t.mom = GeoArgs{tp.tile_m, tp.tile_so, tp.uidx, tp.geo, mm};
    t.defo = GeoArgs{tp.tile_m, tp.tile_so, tp.uidx, tp.geo, md};
    t.mom_bytes = dim == 3 ? (size_t)mm * 36 : (size_t)mm * 16;   // k_tl_mom32g: 9 floats per neighbour in 3D
    t.defo_bytes = (size_t)md * 16;
    // persistent form: both entry buffers, both staging buffers and three lists
    const size_t limit = 220 * 1024;
    int gw = kTileRows * st->plan_maxrow;
    t.pmom = PipeArgs{tp.ntiles, gw, mm, (mm + 3) & ~3};
    t.pdefo = PipeArgs{tp.ntiles, gw, md, (md + 3) & ~3};
    t.pmom_bytes = pipe_smem_bytes(t.pmom, npl);
    t.pdefo_bytes = pipe_smem_bytes(t.pdefo, 1);
    const bool persistent = ctx->tile_pipe == SPH_PIPE_PERSISTENT;
    t.pipe_mom = persistent && t.pmom_bytes <= limit;
    t.pipe_defo = persistent && t.pdefo_bytes <= limit;
    // bulk form of the deformation pass: three blocks per SM, each with its staged
    // neighbours and up to ecap entries in shared memory
    t.bulk_defo = ctx->tile_pipe == SPH_PIPE_BULK;
    if (t.bulk_defo) {
        const size_t per_block = (227 * 1024) / 3 - 1024;
        int64_t room = ((int64_t)per_block - (int64_t)md * 16 - 16) / 16;
        int64_t want = (int64_t)kTileRows * st->plan_maxrow;
        t.defo.tile_e = tp.tile_e;
        t.defo.ecap = (int)std::max<int64_t>(0, std::min(room, want));
        t.bulk_defo = t.defo.ecap > 0;
        t.defo_bytes = (size_t)(md + t.defo.ecap) * 16 + 16;
        t.defo.test_polls = ctx->wait_test_polls;
    }
    // geometry form of the deformation pass: both record halves staged, the slot section
    t.geom_defo = ctx->tile_pipe == SPH_PIPE_GEOM &&
                  st->plan_bytes >= (int64_t)tl_plan_total(n, st->plan_nnz, st->plan_maxrow);
    if (t.geom_defo) {
        int mg = stage_mcap(st->plan_maxm, 2, ctx->stage_cap);
        t.defo.mcap = mg;
        t.defo.slots = reinterpret_cast<const uint16_t*>(reinterpret_cast<const unsigned char*>(st->plan) +
                                                         tl_slot_offset(n, st->plan_nnz, st->plan_maxrow));
        t.defo.spos = reinterpret_cast<const uint16_t*>(reinterpret_cast<const unsigned char*>(st->plan) +
                                                        tl_spos_offset(n, st->plan_nnz, st->plan_maxrow));
        t.defo.sinv = reinterpret_cast<const uint16_t*>(reinterpret_cast<const unsigned char*>(st->plan) +
                                                        tl_sinv_offset(n, st->plan_nnz, st->plan_maxrow));
        // the tile's slot block in shared memory too, up to 128 positions (32 KB)
        t.defo.tile_e = tp.tile_e;
        t.defo.ecap = st->plan_maxrow <= 128 ? (int)st->plan_maxrow : 0;
        t.defo_bytes = (size_t)mg * 32 + (size_t)t.defo.ecap * kTileRows * 2 + 16;   // + the slot copy's mbarrier
        t.defo.test_polls = ctx->wait_test_polls;
        // the momentum pass's geometry form (used on boxes without periodic axes): position
        // and V0_j M_j staged, 48 bytes per neighbour in 3D (24 in 2D); slots and S_i read
        // from the plan
        t.geom_mom = true;
        const int mr = stage_mcap(st->plan_maxm, dim == 3 ? 3 : 2, ctx->stage_cap);
        t.momr = t.defo;
        t.momr.mcap = mr;
        t.momr.wsum = reinterpret_cast<const float4*>(reinterpret_cast<const unsigned char*>(st->plan) +
                                                      tl_wsum_offset(n, st->plan_nnz, st->plan_maxrow));
        t.momr_bytes = dim == 3 ? (size_t)mr * 48 : (size_t)mr * 16 + align16((size_t)mr * 8);
    }
    int64_t g = ctx->num_sms > 0 ? ctx->num_sms : 1;
    t.grid = (int)(g < tp.ntiles ? g : tp.ntiles);
    return t;
}

template <int DIM, int LANES, bool PER>
void tl32_passes(int which, int out, int64_t n, const sph_tlsph_state* st, const TLK<float>& K, double* r1,
                 double* r2, cudaStream_t s) {
    const int block = 256;
    dim3 g(grid_for(n * LANES, block)), b(block);
    if (which == 0) {
        if (out == OUT_RATES)
            k_tl_mom32<DIM, OUT_RATES, LANES, PER><<<g, b, 0, s>>>(st->rm, st->rd, st->row_ptr, st->col, n, K, r1);
        else
            k_tl_mom32<DIM, OUT_STEP, LANES, PER><<<g, b, 0, s>>>(st->rm, st->rd, st->row_ptr, st->col, n, K, nullptr);
    } else {
        if (out == OUT_RATES)
            k_tl_defo32<DIM, OUT_RATES, LANES, PER><<<g, b, 0, s>>>(st->rd, st->rm, st->row_ptr, st->col, n, K,
                                                                   st->B32, st->H32, st->u32, r2);
        else
            k_tl_defo32<DIM, OUT_STEP, LANES, PER><<<g, b, 0, s>>>(st->rd, st->rm, st->row_ptr, st->col, n, K,
                                                                  st->B32, st->H32, st->u32, nullptr);
    }
}

// Bytes of the float32 records: RM (V0, the position code and M: 16 floats in 3D, 8 in 2D)
// and RD (position code and velocity: 8 floats).
static inline size_t tl_rm_bytes(int64_t n, int dim) { return (size_t)n * (dim == 3 ? 64 : 32); }
static inline size_t tl_rd_bytes(int64_t n) { return (size_t)n * 32; }

// hx/ux (a step's deformation pass, OUT_STEP): the caller's host copies of H and u, written
// by the geometry form of the pass itself; returns whether the pass wrote them.
template <int DIM>
bool tl32_plan_pass(sph_ctx* ctx, int which, int out, int64_t n, const sph_tlsph_state* st, const TLK<float>& K,
                    const TlPlan& tp, double* r1, double* r2, cudaStream_t s, bool dependent = true,
                    float* hx = nullptr, float* ux = nullptr) {
    dim3 g((unsigned)((n + kTileRows - 1) / kTileRows)), b(kTileRows), gp((unsigned)tp.grid);
    if (which == 0) {
        if (tp.pipe_mom) {
            ctx->waits_pending = true;
            auto* f = out == OUT_RATES ? k_tl_mom32p<DIM, OUT_RATES> : k_tl_mom32p<DIM, OUT_STEP>;
            sph_allow_dynamic_smem((const void*)f);
            f<<<gp, b, tp.pmom_bytes, s>>>(st->rm, st->rd, st->row_ptr, n, K, tp.mom, tp.pmom,
                                           out == OUT_RATES ? r1 : nullptr, ctx->flags);
        } else if (tp.geom_mom && !K.periodic) {
            // programmatic dependent launch: the pass's plan reads overlap the previous
            // pass's last blocks (a launch error is left to cudaGetLastError)
            auto* f = out == OUT_RATES ? k_tl_mom32r<DIM, OUT_RATES> : k_tl_mom32r<DIM, OUT_STEP>;
            sph_allow_dynamic_smem((const void*)f);
            // the records the pass gathers (RM) kept in L2 between steps
            const L2Win w = sph_l2_window(ctx, st->rm, tl_rm_bytes(n, DIM), tl_rm_bytes(n, DIM) + tl_rd_bytes(n));
            (void)launch_dependent_win(dependent, w, f, g, b, tp.momr_bytes, s, (const float*)st->rm, st->rd,
                                   (const int64_t*)st->row_ptr, n, K, tp.momr, out == OUT_RATES ? r1 : nullptr);
        } else {
            auto* f = out == OUT_RATES ? k_tl_mom32g<DIM, OUT_RATES> : k_tl_mom32g<DIM, OUT_STEP>;
            sph_allow_dynamic_smem((const void*)f);
            f<<<g, b, tp.mom_bytes, s>>>(st->rm, st->rd, st->row_ptr, n, K, tp.mom, out == OUT_RATES ? r1 : nullptr);
        }
    } else {
        if (tp.pipe_defo) {
            ctx->waits_pending = true;
            auto* f = out == OUT_RATES ? k_tl_defo32p<DIM, OUT_RATES> : k_tl_defo32p<DIM, OUT_STEP>;
            sph_allow_dynamic_smem((const void*)f);
            f<<<gp, b, tp.pdefo_bytes, s>>>(st->rd, st->rm, st->row_ptr, n, K, tp.defo, tp.pdefo, st->B32, st->H32,
                                            st->u32, out == OUT_RATES ? r2 : nullptr, ctx->flags);
        } else {
            auto* f = tp.bulk_defo ? (out == OUT_RATES ? k_tl_defo32g<DIM, OUT_RATES, true>
                                                       : k_tl_defo32g<DIM, OUT_STEP, true>)
                                   : (out == OUT_RATES ? k_tl_defo32g<DIM, OUT_RATES, false>
                                                       : k_tl_defo32g<DIM, OUT_STEP, false>);
            const bool host = tp.geom_defo && out == OUT_STEP && hx && ux;
            if (tp.geom_defo) {
                if (K.periodic)
                    f = out == OUT_RATES ? k_tl_defo32g<DIM, OUT_RATES, false, true, true>
                        : host           ? k_tl_defo32g<DIM, OUT_STEP, false, true, true, true>
                                         : k_tl_defo32g<DIM, OUT_STEP, false, true, true>;
                else
                    f = out == OUT_RATES ? k_tl_defo32g<DIM, OUT_RATES, false, true, false>
                        : host           ? k_tl_defo32g<DIM, OUT_STEP, false, true, false, true>
                                         : k_tl_defo32g<DIM, OUT_STEP, false, true, false>;
            }
            if (tp.bulk_defo || tp.geom_defo) ctx->waits_pending = true;
            sph_allow_dynamic_smem((const void*)f);
            // the records the geometry form gathers (RD) kept in L2 between steps
            const L2Win w = tp.geom_defo ? sph_l2_window(ctx, st->rd, tl_rd_bytes(n), tl_rm_bytes(n, DIM) + tl_rd_bytes(n))
                                         : L2Win{};
            if (tp.geom_defo)
                (void)launch_dependent_win(dependent, w, f, g, b, tp.defo_bytes, s, (const float*)st->rd, st->rm,
                                       (const int64_t*)st->row_ptr, n, K, tp.defo, (const float*)st->B32, st->H32,
                                       st->u32, out == OUT_RATES ? r2 : nullptr, ctx->flags, host ? hx : nullptr,
                                       host ? ux : nullptr);
            else
                f<<<g, b, tp.defo_bytes, s>>>(st->rd, st->rm, st->row_ptr, n, K, tp.defo, st->B32, st->H32, st->u32,
                                              out == OUT_RATES ? r2 : nullptr, ctx->flags, nullptr, nullptr);
            return host;
        }
    }
    return false;
}

template <int DIM, bool PER>
void tl32_lanes(int lanes, int which, int out, int64_t n, const sph_tlsph_state* st, const TLK<float>& K,
                double* r1, double* r2, cudaStream_t s) {
    switch (lanes) {
        case 1: tl32_passes<DIM, 1, PER>(which, out, n, st, K, r1, r2, s); break;
        case 2: tl32_passes<DIM, 2, PER>(which, out, n, st, K, r1, r2, s); break;
        case 8: tl32_passes<DIM, 8, PER>(which, out, n, st, K, r1, r2, s); break;
        default: tl32_passes<DIM, 4, PER>(which, out, n, st, K, r1, r2, s); break;
    }
}

// One float32 pass: on the tile plan when the state has one, else the gather form
// with the context's lanes per row.
template <int DIM>
bool tl32(sph_ctx* ctx, int lanes, int which, int out, int64_t n, const sph_tlsph_state* st, const TLK<float>& K,
          const TlPlan& tp, double* r1, double* r2, cudaStream_t s, bool dependent = true, float* hx = nullptr,
          float* ux = nullptr) {
    if (tp.on) return tl32_plan_pass<DIM>(ctx, which, out, n, st, K, tp, r1, r2, s, dependent, hx, ux);
    if (K.periodic) tl32_lanes<DIM, true>(lanes, which, out, n, st, K, r1, r2, s);
    else tl32_lanes<DIM, false>(lanes, which, out, n, st, K, r1, r2, s);
    return false;
}

bool fp32_ready(const sph_tlsph_state* st) { return st->rd && st->rm && st->H32 && st->u32 && st->B32; }
bool fp64_ready(const sph_tlsph_state* st) { return st->x && st->v && st->H && st->M; }

}  // namespace

extern "C" int sph_tlsph_pack(sph_ctx* ctx, const sph_tlsph_params* p, const sph_tlsph_state* st, void* stream) {
    if (!ctx) return SPH_ERR_ARG;
    int r = check_tl(p, st);
    if (r) return r;
    int64_t n = p->dom.n;
    if (n == 0) return SPH_OK;
    if (!fp32_ready(st) || !st->x || !st->v || !st->H) return SPH_ERR_ARG;
    if (((uintptr_t)st->rd & 31u) || ((uintptr_t)st->rm & 31u)) return SPH_ERR_ARG;
    cudaStream_t s = as_stream(stream);
    RelGrid g = make_rel_grid(p->dom);
    if (p->dom.dim == 2)
        k_tl_pack<2><<<grid_for(n, 256), 256, 0, s>>>(st->r0, st->V0, st->B0, st->fixed, st->x, st->v, st->H, n, g,
                                                      st->rd, st->rm, st->H32, st->u32, st->B32);
    else
        k_tl_pack<3><<<grid_for(n, 256), 256, 0, s>>>(st->r0, st->V0, st->B0, st->fixed, st->x, st->v, st->H, n, g,
                                                      st->rd, st->rm, st->H32, st->u32, st->B32);
    SPH_LAUNCH_CHECK(ctx);
    return SPH_OK;
}

// Tile plan of the state's lists and reference configuration (see sph.h).
extern "C" int sph_tlsph_plan(sph_ctx* ctx, const sph_tlsph_params* p, sph_tlsph_state* st, void* stream) {
    if (!ctx) return SPH_ERR_ARG;
    int r = check_tl(p, st);
    if (r) return r;
    if (!st->plan) return SPH_ERR_ARG;
    int64_t n = p->dom.n;
    cudaStream_t s = as_stream(stream);
    st->plan_nnz = 0;
    st->plan_maxm = st->plan_maxrow = 0;
    if (n == 0) return SPH_OK;
    int64_t nnz = 0, maxrow = 0;
    r = sph_row_stats(ctx, st->row_ptr, n, s, &nnz, &maxrow);
    if (r) return r;
    if (st->plan_bytes < (int64_t)tl_plan_total(n, nnz, maxrow)) return SPH_ERR_CAPACITY;
    if (nnz == 0) return SPH_OK;
    int32_t mm = 0, mp = 0, mw = 0;
    r = sph_build_tile_plan(ctx, st->row_ptr, st->col, n, nnz, st->plan, s, &mm, &mp, &mw);
    if (r) return r;
    if (mw != maxrow) return SPH_ERR_ARG;     // both are the longest row of the same lists
    TilePlan tp = tile_plan_view(st->plan, n, nnz);
    uint16_t* slots = reinterpret_cast<uint16_t*>(reinterpret_cast<unsigned char*>(st->plan) +
                                                  tl_slot_offset(n, nnz, maxrow));
    float4* wsum = reinterpret_cast<float4*>(reinterpret_cast<unsigned char*>(st->plan) +
                                             tl_wsum_offset(n, nnz, maxrow));
    uint16_t* spos = reinterpret_cast<uint16_t*>(reinterpret_cast<unsigned char*>(st->plan) +
                                                 tl_spos_offset(n, nnz, maxrow));
    uint16_t* sinv = reinterpret_cast<uint16_t*>(reinterpret_cast<unsigned char*>(st->plan) +
                                                 tl_sinv_offset(n, nnz, maxrow));
    TLK<double> K = make_tl_consts<double>(p);
    unsigned nt = (unsigned)tp.ntiles;
    if (p->dom.dim == 2)
        k_tl_geo<2><<<nt, kTileRows, 0, s>>>(st->r0, st->V0, st->row_ptr, st->col, tp.lcol, tp.tile_m, tp.tile_e,
                                             tp.tile_so, n, K, tp.geo, slots, wsum, spos, sinv);
    else
        k_tl_geo<3><<<nt, kTileRows, 0, s>>>(st->r0, st->V0, st->row_ptr, st->col, tp.lcol, tp.tile_m, tp.tile_e,
                                             tp.tile_so, n, K, tp.geo, slots, wsum, spos, sinv);
    SPH_LAUNCH_CHECK(ctx);
    SPH_CUDA(ctx, cudaStreamSynchronize(s));
    st->plan_nnz = nnz;
    st->plan_maxm = mm;
    st->plan_maxrow = mw;
    return SPH_OK;
}

// Bytes of the tile plan of this state's lists (synchronises the stream).
extern "C" int sph_tlsph_plan_bytes(sph_ctx* ctx, const sph_tlsph_params* p, const sph_tlsph_state* st,
                                    int64_t* bytes_host, void* stream) {
    if (!ctx || !bytes_host) return SPH_ERR_ARG;
    int r = check_tl(p, st);
    if (r) return r;
    int64_t n = p->dom.n, nnz = 0, maxrow = 0;
    if (n > 0) {
        r = sph_row_stats(ctx, st->row_ptr, n, as_stream(stream), &nnz, &maxrow);
        if (r) return r;
    }
    *bytes_host = (int64_t)tl_plan_total(n, nnz, maxrow);
    return SPH_OK;
}

// The float32 form's dynamic state exchanged in float32: u = x - r0, v, H = F - I.
template <int DIM>
__global__ void k_tl_load32(const float* __restrict__ u, const float* __restrict__ v, const float* __restrict__ H,
                            int64_t n, float* __restrict__ RD, float* __restrict__ u32, float* __restrict__ H32) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
        u32[a * n + i] = u[a * n + i];
        RD[8 * i + 4 + a] = v[a * n + i];
    }
#pragma unroll
    for (int k = 0; k < DIM * DIM; ++k) H32[k * n + i] = H[k * n + i];
}

template <int DIM>
__global__ void k_tl_store32(const float* __restrict__ RD, const float* __restrict__ u32,
                             const float* __restrict__ H32, int64_t n, float* __restrict__ u, float* __restrict__ v,
                             float* __restrict__ H) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
        u[a * n + i] = u32[a * n + i];
        v[a * n + i] = RD[8 * i + 4 + a];
    }
#pragma unroll
    for (int k = 0; k < DIM * DIM; ++k) H[k * n + i] = H32[k * n + i];
}

// The pieces of sph_tlsph_step_host32: H and v read in, with the stress factor of the
// read H (as k_tl_stress32); u read in; v written out; H and u written out.
template <int DIM>
__global__ void k_tl_load32_hv(const float* __restrict__ v, const float* __restrict__ H, int64_t n, TLK<float> K,
                               const float* __restrict__ B32, float* __restrict__ RD, float* __restrict__ H32,
                               float* __restrict__ RM) {
    constexpr int NS = DIM == 2 ? 3 : 6;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float h[DIM * DIM], b[NS], m[DIM * DIM];
#pragma unroll
    for (int a = 0; a < DIM; ++a) RD[8 * i + 4 + a] = v[a * n + i];
#pragma unroll
    for (int k = 0; k < DIM * DIM; ++k) {
        h[k] = H[k * n + i];
        H32[k * n + i] = h[k];
    }
#pragma unroll
    for (int q = 0; q < NS; ++q) b[q] = B32[q * n + i];
    stress_factor<DIM, float>(h, b, K, m);
    store_M<DIM>(RM, i, m);
}

template <int DIM>
__global__ void k_tl_store32_v(const float* __restrict__ RD, int64_t n, float* __restrict__ v) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
#pragma unroll
    for (int a = 0; a < DIM; ++a) v[a * n + i] = RD[8 * i + 4 + a];
}

template <int DIM>
__global__ void k_tl_store32_hu(const float* __restrict__ H32, const float* __restrict__ u32, int64_t n,
                                float* __restrict__ H, float* __restrict__ u) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
#pragma unroll
    for (int a = 0; a < DIM; ++a) u[a * n + i] = u32[a * n + i];
#pragma unroll
    for (int k = 0; k < DIM * DIM; ++k) H[k * n + i] = H32[k * n + i];
}

extern "C" int sph_tlsph_load32(sph_ctx* ctx, const sph_tlsph_params* p, const sph_tlsph_state* st, const float* u,
                                const float* v, const float* H, void* stream) {
    if (!ctx) return SPH_ERR_ARG;
    int r = check_tl(p, st);
    if (r) return r;
    const int64_t n = p->dom.n;
    if (n == 0) return SPH_OK;
    if (!u || !v || !H || !st->rd || !st->u32 || !st->H32) return SPH_ERR_ARG;
    cudaStream_t s = as_stream(stream);
    if (p->dom.dim == 2) k_tl_load32<2><<<grid_for(n, 256), 256, 0, s>>>(u, v, H, n, st->rd, st->u32, st->H32);
    else k_tl_load32<3><<<grid_for(n, 256), 256, 0, s>>>(u, v, H, n, st->rd, st->u32, st->H32);
    SPH_LAUNCH_CHECK(ctx);
    return SPH_OK;
}

extern "C" int sph_tlsph_store32(sph_ctx* ctx, const sph_tlsph_params* p, const sph_tlsph_state* st, float* u,
                                 float* v, float* H, void* stream) {
    if (!ctx) return SPH_ERR_ARG;
    int r = check_tl(p, st);
    if (r) return r;
    const int64_t n = p->dom.n;
    if (n == 0) return SPH_OK;
    if (!u || !v || !H || !st->rd || !st->u32 || !st->H32) return SPH_ERR_ARG;
    cudaStream_t s = as_stream(stream);
    if (p->dom.dim == 2) k_tl_store32<2><<<grid_for(n, 256), 256, 0, s>>>(st->rd, st->u32, st->H32, n, u, v, H);
    else k_tl_store32<3><<<grid_for(n, 256), 256, 0, s>>>(st->rd, st->u32, st->H32, n, u, v, H);
    SPH_LAUNCH_CHECK(ctx);
    return SPH_OK;
}

// nsteps float32 steps with the state kept by the caller (sph.h): per step the same
// values as sph_tlsph_load32, sph_tlsph_step(1) and sph_tlsph_store32.  The stress update
// is done by the kernel that reads H in; u is copied in by a copy engine on a second
// stream while the momentum pass runs (only the deformation pass needs it), and v,
// gathered from the records into a device buffer once the momentum pass has made it
// final, is copied out there while the deformation pass runs.  Copy engines, not kernels,
// move these two, so that they take no SM from the passes they overlap; events order the
// two streams, and the caller's stream waits for the second at the end of each step.
namespace {

template <int DIM>
int tl_step_host32(sph_ctx* ctx, const sph_tlsph_params* p, const sph_tlsph_state* st, float* u, float* v,
                   float* H, int nsteps, cudaStream_t s) {
    const int64_t n = p->dom.n;
    if (!ctx->side_stream) SPH_CUDA(ctx, cudaStreamCreateWithFlags(&ctx->side_stream, cudaStreamNonBlocking));
    for (cudaEvent_t& e : ctx->side_ev)
        if (!e) SPH_CUDA(ctx, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    cudaStream_t s2 = ctx->side_stream;
    cudaEvent_t hv_in = ctx->side_ev[0], u_in = ctx->side_ev[1], mom_done = ctx->side_ev[2], v_out = ctx->side_ev[3];
    int r = SPH_OK;
    float* vout = (float*)sph_scratch(ctx, S_TL_VOUT, (size_t)DIM * n * sizeof(float), &r);
    if (r) return r;
    const size_t ubytes = (size_t)DIM * n * sizeof(float);
    TLK<float> K = make_tl_consts<float>(p);
    TlPlan ts = tl_plan(ctx, st, n, DIM);
    const int lanes = ctx->lanes[SPH_PASS_TLSPH];
    const unsigned g = grid_for(n, 256);
    for (int k = 0; k < nsteps; ++k) {
        k_tl_load32_hv<DIM><<<g, 256, 0, s>>>(v, H, n, K, st->B32, st->rd, st->H32, st->rm);
        SPH_CUDA(ctx, cudaEventRecord(hv_in, s));
        SPH_CUDA(ctx, cudaStreamWaitEvent(s2, hv_in, 0));
        SPH_CUDA(ctx, cudaMemcpyAsync(st->u32, u, ubytes, cudaMemcpyDefault, s2));
        SPH_CUDA(ctx, cudaEventRecord(u_in, s2));
        int t = sph_timer_begin(ctx, SPH_TIMER_TL_MOMENTUM, s);
        tl32<DIM>(ctx, lanes, 0, OUT_STEP, n, st, K, ts, nullptr, nullptr, s, false);
        sph_timer_end(ctx, t, s);
        k_tl_store32_v<DIM><<<g, 256, 0, s>>>(st->rd, n, vout);
        SPH_CUDA(ctx, cudaEventRecord(mom_done, s));
        SPH_CUDA(ctx, cudaStreamWaitEvent(s2, mom_done, 0));
        SPH_CUDA(ctx, cudaMemcpyAsync(v, vout, ubytes, cudaMemcpyDefault, s2));
        SPH_CUDA(ctx, cudaEventRecord(v_out, s2));
        SPH_CUDA(ctx, cudaStreamWaitEvent(s, u_in, 0));
        t = sph_timer_begin(ctx, SPH_TIMER_TL_DEFORM, s);
        // the geometry form writes H and u back itself, the write-back overlapping the pass
        const bool direct = tl32<DIM>(ctx, lanes, 1, OUT_STEP, n, st, K, ts, nullptr, nullptr, s, false, H, u);
        sph_timer_end(ctx, t, s);
        if (!direct) k_tl_store32_hu<DIM><<<g, 256, 0, s>>>(st->H32, st->u32, n, H, u);
        // the next step's read of v (and the caller's use of it) after its write-back
        SPH_CUDA(ctx, cudaStreamWaitEvent(s, v_out, 0));
    }
    SPH_LAUNCH_CHECK(ctx);
    return SPH_OK;
}

}  // namespace

extern "C" int sph_tlsph_step_host32(sph_ctx* ctx, const sph_tlsph_params* p, const sph_tlsph_state* st, float* u,
                                     float* v, float* H, int nsteps, void* stream) {
    if (!ctx || nsteps < 0) return SPH_ERR_ARG;
    int r = check_tl(p, st);
    if (r) return r;
    if (p->precision != SPH_FP32_KAHAN || !fp32_ready(st)) return SPH_ERR_ARG;
    const int64_t n = p->dom.n;
    if (n == 0 || nsteps == 0) return SPH_OK;
    if (!u || !v || !H) return SPH_ERR_ARG;
    cudaStream_t s = as_stream(stream);
    return p->dom.dim == 2 ? tl_step_host32<2>(ctx, p, st, u, v, H, nsteps, s)
                           : tl_step_host32<3>(ctx, p, st, u, v, H, nsteps, s);
}

extern "C" int sph_tlsph_unpack(sph_ctx* ctx, const sph_tlsph_params* p, const sph_tlsph_state* st, void* stream) {
    if (!ctx) return SPH_ERR_ARG;
    int r = check_tl(p, st);
    if (r) return r;
    int64_t n = p->dom.n;
    if (n == 0) return SPH_OK;
    if (!st->rd || !st->H32 || !st->u32 || !st->x || !st->v || !st->H) return SPH_ERR_ARG;
    cudaStream_t s = as_stream(stream);
    if (p->dom.dim == 2)
        k_tl_unpack<2><<<grid_for(n, 256), 256, 0, s>>>(st->r0, st->rd, st->H32, st->u32, n, st->x, st->v, st->H);
    else
        k_tl_unpack<3><<<grid_for(n, 256), 256, 0, s>>>(st->r0, st->rd, st->H32, st->u32, n, st->x, st->v, st->H);
    SPH_LAUNCH_CHECK(ctx);
    // a bounded wait that expired in a persistent planned pass since the last unpack
    if (!ctx->waits_pending) return SPH_OK;
    ctx->waits_pending = false;
    return sph_take_timeout(ctx, s);
}

// Kinetic and stored energy of the float64 state, reduced in float64 in a fixed order:
// per block a tree over its 256 particles, then one block over the partials.
// psi: neo-Hookean G/2 (tr C - d) - G ln J + lambda/2 (ln J)^2 (the energy of
// S = G (I - C^-1) + lambda ln J C^-1), SVK lambda/2 (tr E)^2 + G E:E (Eq. 29's law).
template <int DIM>
__global__ void k_tl_energy(const double* __restrict__ V0, const double* __restrict__ v,
                            const double* __restrict__ H, int64_t n, double rho0, double lam, double G, int law,
                            double* __restrict__ partial) {
    __shared__ double sh[2][256];
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double ke = 0.0, pe = 0.0;
    if (i < n) {
        double F[DIM][DIM], C[DIM][DIM];
        for (int a = 0; a < DIM; ++a)
            for (int b = 0; b < DIM; ++b) F[a][b] = (a == b ? 1.0 : 0.0) + H[(a * DIM + b) * n + i];
        double vv = 0.0;
        for (int a = 0; a < DIM; ++a) vv += v[a * n + i] * v[a * n + i];
        for (int a = 0; a < DIM; ++a)
            for (int b = 0; b < DIM; ++b) {
                double c = 0.0;
                for (int k = 0; k < DIM; ++k) c += F[k][a] * F[k][b];
                C[a][b] = c;
            }
        double psi;
        if (law == SPH_NEO_HOOKEAN) {
            double J = DIM == 2 ? F[0][0] * F[1][1] - F[0][1] * F[1][0]
                                : F[0][0] * (F[1][1] * F[2][2] - F[1][2] * F[2][1]) -
                                      F[0][1] * (F[1][0] * F[2][2] - F[1][2] * F[2][0]) +
                                      F[0][2] * (F[1][0] * F[2][1] - F[1][1] * F[2][0]);
            double trC = 0.0;
            for (int a = 0; a < DIM; ++a) trC += C[a][a];
            const double lnJ = log(J);
            psi = 0.5 * G * (trC - DIM) - G * lnJ + 0.5 * lam * lnJ * lnJ;
        } else {
            double trE = 0.0, EE = 0.0;
            for (int a = 0; a < DIM; ++a)
                for (int b = 0; b < DIM; ++b) {
                    const double e = 0.5 * (C[a][b] - (a == b ? 1.0 : 0.0));
                    EE += e * e;
                    if (a == b) trE += e;
                }
            psi = 0.5 * lam * trE * trE + G * EE;
        }
        ke = 0.5 * rho0 * V0[i] * vv;
        pe = V0[i] * psi;
    }
    sh[0][threadIdx.x] = ke;
    sh[1][threadIdx.x] = pe;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) {
            sh[0][threadIdx.x] += sh[0][threadIdx.x + o];
            sh[1][threadIdx.x] += sh[1][threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        partial[2 * blockIdx.x] = sh[0][0];
        partial[2 * blockIdx.x + 1] = sh[1][0];
    }
}

__global__ void k_tl_energy_sum(const double* __restrict__ partial, int nb, double* __restrict__ out) {
    __shared__ double sh[2][256];
    double a = 0.0, b = 0.0;
    for (int k = threadIdx.x; k < nb; k += blockDim.x) {
        a += partial[2 * k];
        b += partial[2 * k + 1];
    }
    sh[0][threadIdx.x] = a;
    sh[1][threadIdx.x] = b;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) {
            sh[0][threadIdx.x] += sh[0][threadIdx.x + o];
            sh[1][threadIdx.x] += sh[1][threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[0] = sh[0][0];
        out[1] = sh[1][0];
    }
}

extern "C" int sph_tlsph_energy(sph_ctx* ctx, const sph_tlsph_params* p, const sph_tlsph_state* st, double* out_host,
                                void* stream) {
    if (!ctx || !out_host) return SPH_ERR_ARG;
    int r = check_tl(p, st);
    if (r) return r;
    out_host[0] = out_host[1] = 0.0;
    const int64_t n = p->dom.n;
    if (n == 0) return SPH_OK;
    if (!st->v || !st->H || !st->V0) return SPH_ERR_ARG;
    cudaStream_t s = as_stream(stream);
    const int nb = (int)grid_for(n, 256);
    double* partial = (double*)sph_scratch(ctx, S_RED_PARTIAL, (size_t)nb * 16 + 64, &r);
    if (r) return r;
    double* out_d = partial + 2 * (size_t)nb;
    if (p->dom.dim == 2)
        k_tl_energy<2><<<nb, 256, 0, s>>>(st->V0, st->v, st->H, n, p->rho0, p->lambda, p->G, p->law, partial);
    else
        k_tl_energy<3><<<nb, 256, 0, s>>>(st->V0, st->v, st->H, n, p->rho0, p->lambda, p->G, p->law, partial);
    k_tl_energy_sum<<<1, 256, 0, s>>>(partial, nb, out_d);
    SPH_LAUNCH_CHECK(ctx);
    double* hp = (double*)ctx->pinned;
    SPH_CUDA(ctx, cudaMemcpyAsync(hp + 48, out_d, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
    SPH_CUDA(ctx, cudaStreamSynchronize(s));
    if (!isfinite(hp[48]) || !isfinite(hp[49])) return SPH_ERR_NONFINITE;
    out_host[0] = hp[48];
    out_host[1] = hp[49];
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
        TlPlan ts = tl_plan(ctx, st, n, dim);
        int lanes = ctx->lanes[SPH_PASS_TLSPH];
        if (dim == 2) {
            k_tl_stress32<2><<<grid_for(n, 128), 128, 0, s>>>(st->H32, st->B32, n, K, st->rm);
            tl32<2>(ctx, lanes, 0, OUT_RATES, n, st, K, ts, dvdt, dFdt, s);
            tl32<2>(ctx, lanes, 1, OUT_RATES, n, st, K, ts, dvdt, dFdt, s);
        } else {
            k_tl_stress32<3><<<grid_for(n, 128), 128, 0, s>>>(st->H32, st->B32, n, K, st->rm);
            tl32<3>(ctx, lanes, 0, OUT_RATES, n, st, K, ts, dvdt, dFdt, s);
            tl32<3>(ctx, lanes, 1, OUT_RATES, n, st, K, ts, dvdt, dFdt, s);
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
    TlPlan ts = tl_plan(ctx, st, n, dim);
    int lanes = ctx->lanes[SPH_PASS_TLSPH];
    int t = sph_timer_begin(ctx, SPH_TIMER_TL_STRESS, s);
    if (dim == 2) k_tl_stress32<2><<<grid_for(n, 128), 128, 0, s>>>(st->H32, st->B32, n, K, st->rm);
    else k_tl_stress32<3><<<grid_for(n, 128), 128, 0, s>>>(st->H32, st->B32, n, K, st->rm);
    sph_timer_end(ctx, t, s);
    for (int k = 0; k < nsteps; ++k) {
        t = sph_timer_begin(ctx, SPH_TIMER_TL_MOMENTUM, s);
        if (dim == 2) tl32<2>(ctx, lanes, 0, OUT_STEP, n, st, K, ts, nullptr, nullptr, s);
        else tl32<3>(ctx, lanes, 0, OUT_STEP, n, st, K, ts, nullptr, nullptr, s);
        sph_timer_end(ctx, t, s);
        t = sph_timer_begin(ctx, SPH_TIMER_TL_DEFORM, s);
        if (dim == 2) tl32<2>(ctx, lanes, 1, OUT_STEP, n, st, K, ts, nullptr, nullptr, s);
        else tl32<3>(ctx, lanes, 1, OUT_STEP, n, st, K, ts, nullptr, nullptr, s);
        sph_timer_end(ctx, t, s);
    }
    SPH_LAUNCH_CHECK(ctx);
    return SPH_OK;
}

// Autotuner of the float32 pair passes: times trial_steps steps for each lanes
// setting in {1, 2, 4, 8} on the caller's state, restores the state after each
// trial, and keeps the fastest setting in the context.
extern "C" int sph_autotune_tlsph(sph_ctx* ctx, const sph_tlsph_params* p, const sph_tlsph_state* st,
                                  int trial_steps, int* lanes_host, double* ms_host, void* stream) {
    if (!ctx || trial_steps < 1) return SPH_ERR_ARG;
    int r = check_tl(p, st);
    if (r) return r;
    if (p->precision != SPH_FP32_KAHAN || !fp32_ready(st)) return SPH_ERR_ARG;
    int64_t n = p->dom.n;
    if (n == 0) return SPH_OK;
    int dim = p->dom.dim;
    cudaStream_t s = as_stream(stream);
    size_t brd = (size_t)n * 8 * 4, brm = (size_t)n * (dim == 3 ? 16 : 8) * 4;
    size_t bh = (size_t)n * dim * dim * 4, bu = (size_t)n * dim * 4;
    unsigned char* save = (unsigned char*)sph_scratch(ctx, S_MISC3, brd + brm + bh + bu, &r);
    if (r) return r;
    SPH_CUDA(ctx, cudaMemcpyAsync(save, st->rd, brd, cudaMemcpyDeviceToDevice, s));
    SPH_CUDA(ctx, cudaMemcpyAsync(save + brd, st->rm, brm, cudaMemcpyDeviceToDevice, s));
    SPH_CUDA(ctx, cudaMemcpyAsync(save + brd + brm, st->H32, bh, cudaMemcpyDeviceToDevice, s));
    SPH_CUDA(ctx, cudaMemcpyAsync(save + brd + brm + bh, st->u32, bu, cudaMemcpyDeviceToDevice, s));
    cudaEvent_t e0, e1;
    SPH_CUDA(ctx, cudaEventCreate(&e0));
    SPH_CUDA(ctx, cudaEventCreate(&e1));
    const int lanes_set[4] = {1, 2, 4, 8};
    int keep = ctx->lanes[SPH_PASS_TLSPH];
    const int timing = ctx->timing;
    ctx->timing = 0;
    double best = 1e300;
    int bl = keep;
    for (int li = 0; li < 4; ++li) {
        ctx->lanes[SPH_PASS_TLSPH] = lanes_set[li];
        r = sph_tlsph_step(ctx, p, st, 1, stream);                  // warm
        if (r) break;
        SPH_CUDA(ctx, cudaEventRecord(e0, s));
        r = sph_tlsph_step(ctx, p, st, trial_steps, stream);
        if (r) break;
        SPH_CUDA(ctx, cudaEventRecord(e1, s));
        SPH_CUDA(ctx, cudaEventSynchronize(e1));
        float ms = 0.0f;
        SPH_CUDA(ctx, cudaEventElapsedTime(&ms, e0, e1));
        if (ms < best) { best = ms; bl = lanes_set[li]; }
        SPH_CUDA(ctx, cudaMemcpyAsync(st->rd, save, brd, cudaMemcpyDeviceToDevice, s));
        SPH_CUDA(ctx, cudaMemcpyAsync(st->rm, save + brd, brm, cudaMemcpyDeviceToDevice, s));
        SPH_CUDA(ctx, cudaMemcpyAsync(st->H32, save + brd + brm, bh, cudaMemcpyDeviceToDevice, s));
        SPH_CUDA(ctx, cudaMemcpyAsync(st->u32, save + brd + brm + bh, bu, cudaMemcpyDeviceToDevice, s));
    }
    ctx->timing = timing;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (r) { ctx->lanes[SPH_PASS_TLSPH] = keep; return r; }
    ctx->lanes[SPH_PASS_TLSPH] = bl;
    if (lanes_host) *lanes_host = bl;
    if (ms_host) *ms_host = best / trial_steps;
    SPH_CUDA(ctx, cudaStreamSynchronize(s));
    return SPH_OK;
}
