// x2: Riemann-based Eulerian SPH for compressible flow (Sec. 3.1): the mass, momentum
// and energy rows of Eq. 18 with the ideal-gas EOS (Eqs. 15-16) and the HLLC solver with
// the dissipation limiter (Eqs. 20-24), forward Euler in time.  Readings (see
// include/sph.h): the star density and energy use the normal velocity u where |v| is
// printed; the limited p* adds the two impedance terms; the interface state follows the
// wave fan, the star state when S_l and S_r cross, the star mean at u* = 0.
//
// Two forms:
//  * float64 (the reference form): one thread per particle over its CSR row, the pair
//    geometry evaluated per pair, rates then update;
//  * float32 + compensated sums: particles never move, so every pair's geometry
//    G_ij = -2 V_j (B_i + B_j)/2 grad W_ij and n = -r_ij/r is computed once in float64
//    (sph_compressible_plan) and stored rounded to float32 in a sliced layout (pair k of
//    row i at (i/32)*32*W + 32k + i%32, W the longest row), so the 32 threads of a warp
//    read 32 consecutive entries.  A step is one kernel: each thread reads its
//    neighbours' float32 records (rho, v, p, c, E) from one buffer, evaluates the fluxes,
//    advances its own float64 state and writes its record for the next step into the
//    other buffer.
#include "tiles.cuh"

namespace {

struct CompK {
    double gamma, eta, coef, inv_h, dt;
    double len[3], half[3];
    uint32_t periodic;
};

template <int DIM, typename T>
struct Prim {
    T rho, v[DIM], p, c, E;
};

template <int DIM>
__device__ __forceinline__ Prim<DIM, double> prim(const double* rho, const double* mom, const double* E, int64_t n,
                                                  int64_t i, double gamma) {
    Prim<DIM, double> s;
    s.rho = rho[i];
    double v2 = 0.0;
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
        s.v[a] = mom[a * n + i] / s.rho;
        v2 += s.v[a] * s.v[a];
    }
    s.E = E[i];
    s.p = (gamma - 1.0) * (s.E - 0.5 * s.rho * v2);
    s.c = sqrt(gamma * s.p / s.rho);
    return s;
}

// Interface state (rho_s, v_s, E_s, p_s) of the limited HLLC solver along nrm (i -> j),
// in the arithmetic type T.
template <int DIM, typename T>
__device__ __forceinline__ void hllc(const Prim<DIM, T>& L, const Prim<DIM, T>& R, const T* nrm, T eta, T& rho_s,
                                     T* v_s, T& E_s, T& p_s) {
    const T zero = T(0), half = T(0.5), one = T(1);
    T ul = zero, ur = zero;
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
        ul += L.v[a] * nrm[a];
        ur += R.v[a] * nrm[a];
    }
    const T sl = ul - L.c, sr = ur + R.c;
    const T cbar = half * (L.c + R.c);
    const T beta = fmin(eta * fmax((ul - ur) / cbar, zero), one);
    const T zl = L.rho * L.c, zr = R.rho * R.c;
    const T ustar = (zl * ul + zr * ur + beta * beta * (L.p - R.p)) / (zl + zr);
    const T pstar = half * (L.p + R.p) + half * beta * (zr * (ustar - ur) + zl * (ul - ustar));
    const bool left = sl >= zero && sr > zero;
    const bool right = sr <= zero && sl < zero;
    if (left) {
        rho_s = L.rho;
        E_s = L.E;
        p_s = L.p;
#pragma unroll
        for (int a = 0; a < DIM; ++a) v_s[a] = L.v[a];
        return;
    }
    if (right) {
        rho_s = R.rho;
        E_s = R.E;
        p_s = R.p;
#pragma unroll
        for (int a = 0; a < DIM; ++a) v_s[a] = R.v[a];
        return;
    }
    const T rho_sl = L.rho * (sl - ul) / (sl - ustar);
    const T rho_sr = R.rho * (sr - ur) / (sr - ustar);
    const T E_sl = ((sl - ul) * L.E - L.p * ul + pstar * ustar) / (sl - ustar);
    const T E_sr = ((sr - ur) * R.E - R.p * ur + pstar * ustar) / (sr - ustar);
    if (ustar > zero) { rho_s = rho_sl; E_s = E_sl; }
    else if (ustar < zero) { rho_s = rho_sr; E_s = E_sr; }
    else { rho_s = half * (rho_sl + rho_sr); E_s = half * (E_sl + E_sr); }
    p_s = pstar;
#pragma unroll
    for (int a = 0; a < DIM; ++a) v_s[a] = ustar * nrm[a] + half * (L.v[a] + R.v[a]) - half * (ul + ur) * nrm[a];
}

template <int DIM>
__global__ void k_comp_rates64(const double* __restrict__ pos, const double* __restrict__ vol,
                               const double* __restrict__ B, const int64_t* __restrict__ row_ptr,
                               const int32_t* __restrict__ col, const double* __restrict__ rho,
                               const double* __restrict__ mom, const double* __restrict__ E, int64_t n, CompK K,
                               double* __restrict__ drho, double* __restrict__ dmom, double* __restrict__ dE) {
    constexpr int NS = DIM == 2 ? 3 : 6;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double xi[DIM], Bi[NS];
#pragma unroll
    for (int a = 0; a < DIM; ++a) xi[a] = pos[a * n + i];
#pragma unroll
    for (int t = 0; t < NS; ++t) Bi[t] = B[t * n + i];
    const Prim<DIM, double> Pi = prim<DIM>(rho, mom, E, n, i, K.gamma);
    double sm = 0.0, se = 0.0, sp[DIM];
#pragma unroll
    for (int a = 0; a < DIM; ++a) sp[a] = 0.0;
    for (int64_t p = row_ptr[i], e = row_ptr[i + 1]; p < e; ++p) {
        const int j = col[p];
        double r[DIM], d2 = 0.0;
#pragma unroll
        for (int a = 0; a < DIM; ++a) {
            double dx = xi[a] - pos[a * n + j];
            if ((K.periodic >> a) & 1u) {
                if (dx > K.half[a]) dx -= K.len[a];
                else if (dx < -K.half[a]) dx += K.len[a];
            }
            r[a] = dx;
            d2 += dx * dx;
        }
        const double rr = sqrt(d2);
        const double gs = wendland_gs<double>(rr * K.inv_h, K.coef);
        double gw[DIM], Bb[NS], g[DIM], nrm[DIM];
#pragma unroll
        for (int a = 0; a < DIM; ++a) {
            gw[a] = gs * r[a];
            nrm[a] = -r[a] / rr;
        }
#pragma unroll
        for (int t = 0; t < NS; ++t) Bb[t] = 0.5 * (Bi[t] + B[t * n + j]);
        if (DIM == 2) {
            g[0] = Bb[0] * gw[0] + Bb[1] * gw[1];
            g[1] = Bb[1] * gw[0] + Bb[2] * gw[1];
        } else {
            g[0] = Bb[0] * gw[0] + Bb[1] * gw[1] + Bb[2] * gw[DIM - 1];
            g[1] = Bb[1] * gw[0] + Bb[3] * gw[1] + Bb[4] * gw[DIM - 1];
            g[DIM - 1] = Bb[2] * gw[0] + Bb[4] * gw[1] + Bb[5] * gw[DIM - 1];
        }
        const Prim<DIM, double> Pj = prim<DIM>(rho, mom, E, n, j, K.gamma);
        double rho_s, v_s[DIM], E_s, p_s;
        hllc<DIM, double>(Pi, Pj, nrm, K.eta, rho_s, v_s, E_s, p_s);
        double vg = 0.0;
#pragma unroll
        for (int a = 0; a < DIM; ++a) vg += v_s[a] * g[a];
        const double w = vol[j];
        sm += w * rho_s * vg;
#pragma unroll
        for (int a = 0; a < DIM; ++a) sp[a] += w * (rho_s * v_s[a] * vg + p_s * g[a]);
        se += w * (E_s + p_s) * vg;
    }
    drho[i] = -2.0 * sm;
#pragma unroll
    for (int a = 0; a < DIM; ++a) dmom[a * n + i] = -2.0 * sp[a];
    dE[i] = -2.0 * se;
}

__global__ void k_comp_update(double* __restrict__ rho, double* __restrict__ mom, double* __restrict__ E,
                              const double* __restrict__ drho, const double* __restrict__ dmom,
                              const double* __restrict__ dE, int64_t n, int dim, double dt) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    rho[i] += dt * drho[i];
    for (int a = 0; a < dim; ++a) mom[a * n + i] += dt * dmom[a * n + i];
    E[i] += dt * dE[i];
}

// ------------------------------------------------------------- float32 form
// Plan: plane A float4 [E] (G_x, G_y, n_x, n_y) in 2D, (G_x, G_y, G_z, n_x) in 3D;
// plane B int32 [E] (j) in 2D, float4 [E] (n_y, n_z, j as bits, 0) in 3D; E = number of
// 32-row slices x 32 x W.  Entries past a row's length are never read.
template <int DIM>
constexpr size_t plane_b_bytes() { return DIM == 2 ? 4 : 16; }

static inline int64_t plan_entries(int64_t n, int64_t width) { return (n + 31) / 32 * 32 * width; }

static inline size_t plan_bytes_for(int dim, int64_t n, int64_t width) {
    const int64_t e = plan_entries(n, width);
    return (size_t)e * 16 + (size_t)e * (dim == 2 ? 4 : 16);
}

__device__ __forceinline__ int64_t slot(int64_t i, int k, int width) {
    return (i >> 5) * 32 * (int64_t)width + 32 * (int64_t)k + (i & 31);
}

template <int DIM>
__global__ void k_comp_geo(const double* __restrict__ pos, const double* __restrict__ vol,
                           const double* __restrict__ B, const int64_t* __restrict__ row_ptr,
                           const int32_t* __restrict__ col, int64_t n, CompK K, int width, float4* __restrict__ ga,
                           void* __restrict__ gb) {
    constexpr int NS = DIM == 2 ? 3 : 6;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double xi[DIM], Bi[NS];
#pragma unroll
    for (int a = 0; a < DIM; ++a) xi[a] = pos[a * n + i];
#pragma unroll
    for (int t = 0; t < NS; ++t) Bi[t] = B[t * n + i];
    const int64_t b = row_ptr[i];
    const int len = (int)(row_ptr[i + 1] - b);
    for (int k = 0; k < len; ++k) {
        const int j = col[b + k];
        double r[DIM], d2 = 0.0;
#pragma unroll
        for (int a = 0; a < DIM; ++a) {
            double dx = xi[a] - pos[a * n + j];
            if ((K.periodic >> a) & 1u) {
                if (dx > K.half[a]) dx -= K.len[a];
                else if (dx < -K.half[a]) dx += K.len[a];
            }
            r[a] = dx;
            d2 += dx * dx;
        }
        const double rr = sqrt(d2);
        const double gs = wendland_gs<double>(rr * K.inv_h, K.coef);
        double gw[DIM], Bb[NS], g[DIM], nrm[DIM];
#pragma unroll
        for (int a = 0; a < DIM; ++a) {
            gw[a] = gs * r[a];
            nrm[a] = -r[a] / rr;
        }
#pragma unroll
        for (int t = 0; t < NS; ++t) Bb[t] = 0.5 * (Bi[t] + B[t * n + j]);
        if (DIM == 2) {
            g[0] = Bb[0] * gw[0] + Bb[1] * gw[1];
            g[1] = Bb[1] * gw[0] + Bb[2] * gw[1];
        } else {
            g[0] = Bb[0] * gw[0] + Bb[1] * gw[1] + Bb[2] * gw[DIM - 1];
            g[1] = Bb[1] * gw[0] + Bb[3] * gw[1] + Bb[4] * gw[DIM - 1];
            g[DIM - 1] = Bb[2] * gw[0] + Bb[4] * gw[1] + Bb[5] * gw[DIM - 1];
        }
        const double f = -2.0 * vol[j];
        const int64_t e = slot(i, k, width);
        if (DIM == 2) {
            ga[e] = make_float4((float)(f * g[0]), (float)(f * g[1]), (float)nrm[0], (float)nrm[1]);
            reinterpret_cast<int32_t*>(gb)[e] = j;
        } else {
            ga[e] = make_float4((float)(f * g[0]), (float)(f * g[1]), (float)(f * g[DIM - 1]), (float)nrm[0]);
            reinterpret_cast<float4*>(gb)[e] =
                make_float4((float)nrm[1], (float)nrm[DIM - 1], __int_as_float(j), 0.0f);
        }
    }
}

// float32 record of a particle's state: rec0 = (rho, v_x, v_y, p) in 2D, (rho, v_x, v_y,
// v_z) in 3D; rec1 = (c, E, 0, 0) in 2D, (p, c, E, 0) in 3D.
template <int DIM>
__device__ __forceinline__ void make_rec(float rho, const float* mom, float E, float gamma, float4& r0, float4& r1) {
    const float inv = 1.0f / rho;
    float v[DIM], v2 = 0.0f;
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
        v[a] = mom[a] * inv;
        v2 += v[a] * v[a];
    }
    const float p = (gamma - 1.0f) * (E - 0.5f * rho * v2);
    const float c = sqrtf(gamma * p * inv);
    if (DIM == 2) {
        r0 = make_float4(rho, v[0], v[1], p);
        r1 = make_float4(c, E, 0.0f, 0.0f);
    } else {
        r0 = make_float4(rho, v[0], v[1], v[DIM - 1]);
        r1 = make_float4(p, c, E, 0.0f);
    }
}

template <int DIM>
__device__ __forceinline__ Prim<DIM, float> load_rec(const float4* __restrict__ r0, const float4* __restrict__ r1,
                                                     int64_t j) {
    const float4 a = __ldg(r0 + j), b = __ldg(r1 + j);
    Prim<DIM, float> s;
    s.rho = a.x;
    s.v[0] = a.y;
    s.v[1] = a.z;
    if (DIM == 2) {
        s.p = a.w;
        s.c = b.x;
        s.E = b.y;
    } else {
        s.v[DIM - 1] = a.w;
        s.p = b.x;
        s.c = b.y;
        s.E = b.z;
    }
    return s;
}

template <int DIM>
__global__ void k_comp_rec(const double* __restrict__ rho, const double* __restrict__ mom,
                           const double* __restrict__ E, int64_t n, float gamma, float4* __restrict__ r0,
                           float4* __restrict__ r1) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float m[DIM];
#pragma unroll
    for (int a = 0; a < DIM; ++a) m[a] = (float)mom[a * n + i];
    make_rec<DIM>((float)rho[i], m, (float)E[i], gamma, r0[i], r1[i]);
}

// The float32 solver: the same interface state as hllc<DIM, T>, without branches (the
// wave-fan choice by selects, so the threads of a warp stay converged) and with the
// divisions by cbar, Z_l + Z_r and S_k - u* as approximate reciprocals (rcp.approx, a
// relative error of about 1e-7, well inside the float32 form's tolerance).
__device__ __forceinline__ float rcp_approx(float x) { return __fdividef(1.0f, x); }

template <int DIM>
__device__ __forceinline__ void hllc32(const Prim<DIM, float>& L, const Prim<DIM, float>& R, const float* nrm,
                                       float eta, float& rho_s, float* v_s, float& E_s, float& p_s) {
    float ul = 0.0f, ur = 0.0f;
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
        ul += L.v[a] * nrm[a];
        ur += R.v[a] * nrm[a];
    }
    const float sl = ul - L.c, sr = ur + R.c;
    const float beta = fminf(eta * fmaxf((ul - ur) * rcp_approx(0.5f * (L.c + R.c)), 0.0f), 1.0f);
    const float zl = L.rho * L.c, zr = R.rho * R.c;
    const float ustar = (zl * ul + zr * ur + beta * beta * (L.p - R.p)) * rcp_approx(zl + zr);
    const float pstar = 0.5f * (L.p + R.p) + 0.5f * beta * (zr * (ustar - ur) + zl * (ul - ustar));
    const float il = rcp_approx(sl - ustar), ir = rcp_approx(sr - ustar);
    const float rho_sl = L.rho * (sl - ul) * il, rho_sr = R.rho * (sr - ur) * ir;
    const float pu = pstar * ustar;
    const float E_sl = ((sl - ul) * L.E - L.p * ul + pu) * il;
    const float E_sr = ((sr - ur) * R.E - R.p * ur + pu) * ir;
    float rs = ustar > 0.0f ? rho_sl : (ustar < 0.0f ? rho_sr : 0.5f * (rho_sl + rho_sr));
    float es = ustar > 0.0f ? E_sl : (ustar < 0.0f ? E_sr : 0.5f * (E_sl + E_sr));
    float ps = pstar;
    const float ut = ustar - 0.5f * (ul + ur);
    float vs[DIM];
#pragma unroll
    for (int a = 0; a < DIM; ++a) vs[a] = ut * nrm[a] + 0.5f * (L.v[a] + R.v[a]);
    const bool left = sl >= 0.0f && sr > 0.0f;
    const bool right = sr <= 0.0f && sl < 0.0f;
    rs = left ? L.rho : (right ? R.rho : rs);
    es = left ? L.E : (right ? R.E : es);
    ps = left ? L.p : (right ? R.p : ps);
#pragma unroll
    for (int a = 0; a < DIM; ++a) v_s[a] = left ? L.v[a] : (right ? R.v[a] : vs[a]);
    rho_s = rs;
    E_s = es;
    p_s = ps;
}

// Pair k's plan entry: G (with -2 V_j), the normal and j.
template <int DIM>
__device__ __forceinline__ int load_entry(const float4* __restrict__ ga, const void* __restrict__ gb, int64_t e,
                                          float* G, float* nrm) {
    const float4 a = __ldg(ga + e);
    if (DIM == 2) {
        G[0] = a.x;
        G[1] = a.y;
        nrm[0] = a.z;
        nrm[1] = a.w;
        return __ldg(reinterpret_cast<const int32_t*>(gb) + e);
    } else {
        const float4 b = __ldg(reinterpret_cast<const float4*>(gb) + e);
        G[0] = a.x;
        G[1] = a.y;
        G[DIM - 1] = a.z;
        nrm[0] = a.w;
        nrm[1] = b.x;
        nrm[DIM - 1] = b.y;
        return __float_as_int(b.z);
    }
}

// One pass over the plan, LANES consecutive lanes per row (pairs k = lane, lane + LANES,
// ...), their partial sums combined with shuffles.  UPDATE: advance the float64 state of
// row i by dt and write its next record (n0, n1); otherwise write the rates.  Sums:
// compensated, in pairs (mass, energy), (momentum x, y), (momentum z).
template <int DIM, bool UPDATE, int LANES>
__global__ void __launch_bounds__(128) k_comp32(const float4* __restrict__ r0, const float4* __restrict__ r1,
                                                const float4* __restrict__ ga, const void* __restrict__ gb,
                                                const int64_t* __restrict__ row_ptr, int64_t n, int width,
                                                float gamma, float eta, double dt, double* __restrict__ rho,
                                                double* __restrict__ mom, double* __restrict__ E,
                                                float4* __restrict__ n0, float4* __restrict__ n1) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t i = t / LANES;
    const int lane = (int)(t % LANES);
    // the lanes of a row are all in range or all out of it; out of range they only take
    // part in the shuffles
    const bool active = i < n;
    const Prim<DIM, float> Pi = load_rec<DIM>(r0, r1, active ? i : 0);
    // a plan of other lists is wrong but never read past: rows are cut at its width
    const int len = active ? min((int)(row_ptr[i + 1] - row_ptr[i]), width) : 0;
    const int cnt = len > lane ? (len - lane + LANES - 1) / LANES : 0;
    constexpr int64_t kStride = 32 * LANES;
    Kahan2 me, mxy, mz;
    me.init();
    mxy.init();
    mz.init();
    // software pipeline: while pair m is evaluated, pair m + 1's neighbour record and
    // pair m + 2's plan entry are in flight (the record load then never waits on the
    // entry load of the same iteration)
    int64_t e = active ? slot(i, lane, width) : 0;
    float G1[DIM], N1[DIM], G2[DIM] = {}, N2[DIM] = {};
    int j2 = 0;
    Prim<DIM, float> P1;
    // a plan of other lists reads wrong but in-bounds records: j is clamped to [0, n)
    if (cnt > 0) P1 = load_rec<DIM>(r0, r1, min(max(load_entry<DIM>(ga, gb, e, G1, N1), 0), (int)(n - 1)));
    if (cnt > 1) j2 = load_entry<DIM>(ga, gb, e + kStride, G2, N2);
    e += 2 * kStride;
    for (int m = 0; m < cnt; ++m) {
        float G[DIM], nrm[DIM];
#pragma unroll
        for (int d = 0; d < DIM; ++d) {
            G[d] = G1[d];
            nrm[d] = N1[d];
            G1[d] = G2[d];
            N1[d] = N2[d];
        }
        const Prim<DIM, float> Pj = P1;
        if (m + 1 < cnt) P1 = load_rec<DIM>(r0, r1, min(max(j2, 0), (int)(n - 1)));
        if (m + 2 < cnt) j2 = load_entry<DIM>(ga, gb, e, G2, N2);
        e += kStride;
        float rho_s, v_s[DIM], E_s, p_s;
        hllc32<DIM>(Pi, Pj, nrm, eta, rho_s, v_s, E_s, p_s);
        float vg = 0.0f;
#pragma unroll
        for (int d = 0; d < DIM; ++d) vg += v_s[d] * G[d];
        const float fm = rho_s * vg;
        me.add(make_float2(fm, (E_s + p_s) * vg));
        mxy.add(make_float2(fm * v_s[0] + p_s * G[0], fm * v_s[1] + p_s * G[1]));
        if (DIM == 3) mz.add(make_float2(fm * v_s[DIM - 1] + p_s * G[DIM - 1], 0.0f));
    }
    float2 se = me.value(), sxy = mxy.value(), sz = mz.value();
#pragma unroll
    for (int o = LANES / 2; o > 0; o >>= 1) {
        se.x += __shfl_xor_sync(0xffffffffu, se.x, o);
        se.y += __shfl_xor_sync(0xffffffffu, se.y, o);
        sxy.x += __shfl_xor_sync(0xffffffffu, sxy.x, o);
        sxy.y += __shfl_xor_sync(0xffffffffu, sxy.y, o);
        if (DIM == 3) sz.x += __shfl_xor_sync(0xffffffffu, sz.x, o);
    }
    if (!active || lane != 0) return;
    const float sp[3] = {sxy.x, sxy.y, sz.x};
    if (UPDATE) {
        const double rn = rho[i] + dt * (double)se.x;
        const double En = E[i] + dt * (double)se.y;
        float mf[DIM];
#pragma unroll
        for (int d = 0; d < DIM; ++d) {
            const double m = mom[d * n + i] + dt * (double)sp[d];
            mom[d * n + i] = m;
            mf[d] = (float)m;
        }
        rho[i] = rn;
        E[i] = En;
        make_rec<DIM>((float)rn, mf, (float)En, gamma, n0[i], n1[i]);
    } else {
        rho[i] = (double)se.x;          // the rate outputs
        E[i] = (double)se.y;
#pragma unroll
        for (int d = 0; d < DIM; ++d) mom[d * n + i] = (double)sp[d];
    }
}

int check(const sph_compressible_params* p, const sph_compressible_state* st) {
    if (!p || !st) return SPH_ERR_ARG;
    int r = sph_check_domain(&p->dom);
    if (r) return r;
    if (p->precision != SPH_FP64 && p->precision != SPH_FP32_KAHAN) return SPH_ERR_ARG;
    if (!(p->gamma > 1.0) || !(p->eta >= 0.0) || !(p->dt >= 0.0)) return SPH_ERR_ARG;
    if (p->dom.n > 0 && (!st->row_ptr || !st->col || !st->pos || !st->vol || !st->B || !st->rho || !st->mom ||
                         !st->E))
        return SPH_ERR_ARG;
    return SPH_OK;
}

// The float32 form needs a plan of at least its width's size.
int check_plan(const sph_compressible_params* p, const sph_compressible_state* st) {
    if (p->precision != SPH_FP32_KAHAN || p->dom.n == 0) return SPH_OK;
    if (!st->plan || ((uintptr_t)st->plan & 15u) || st->plan_width < 1) return SPH_ERR_ARG;
    if (st->plan_bytes < (int64_t)plan_bytes_for(p->dom.dim, p->dom.n, st->plan_width)) return SPH_ERR_CAPACITY;
    return SPH_OK;
}

CompK consts(const sph_compressible_params* p) {
    CompK K;
    const int d = p->dom.dim;
    const double h = p->dom.h;
    const double hd2 = d == 2 ? h * h * h * h : h * h * h * h * h;
    K.gamma = p->gamma;
    K.eta = p->eta;
    K.coef = -5.0 * wendland_alpha(d) / hd2;
    K.inv_h = 1.0 / h;
    K.dt = p->dt;
    for (int a = 0; a < 3; ++a) { K.len[a] = p->dom.len[a]; K.half[a] = 0.5 * p->dom.len[a]; }
    K.periodic = p->dom.periodic_mask;
    return K;
}

void launch_rates(const sph_compressible_params* p, const sph_compressible_state* st, const CompK& K, double* drho,
                  double* dmom, double* dE, cudaStream_t s) {
    const int64_t n = p->dom.n;
    if (p->dom.dim == 2)
        k_comp_rates64<2><<<grid_for(n, 128), 128, 0, s>>>(st->pos, st->vol, st->B, st->row_ptr, st->col, st->rho,
                                                           st->mom, st->E, n, K, drho, dmom, dE);
    else
        k_comp_rates64<3><<<grid_for(n, 128), 128, 0, s>>>(st->pos, st->vol, st->B, st->row_ptr, st->col, st->rho,
                                                           st->mom, st->E, n, K, drho, dmom, dE);
}

struct Plan32 {
    const float4* ga;
    const void* gb;
};

Plan32 plan_view(const sph_compressible_state* st, int dim, int64_t n) {
    Plan32 v;
    v.ga = reinterpret_cast<const float4*>(st->plan);
    v.gb = reinterpret_cast<const unsigned char*>(st->plan) + plan_entries(n, st->plan_width) * 16;
    (void)dim;
    return v;
}

// The float32 records of the state into (r0, r1), n float4 each.
void launch_rec(const sph_compressible_params* p, const sph_compressible_state* st, float4* r0, float4* r1,
                cudaStream_t s) {
    const int64_t n = p->dom.n;
    if (p->dom.dim == 2)
        k_comp_rec<2><<<grid_for(n, 256), 256, 0, s>>>(st->rho, st->mom, st->E, n, (float)p->gamma, r0, r1);
    else
        k_comp_rec<3><<<grid_for(n, 256), 256, 0, s>>>(st->rho, st->mom, st->E, n, (float)p->gamma, r0, r1);
}

template <int DIM, bool UPDATE, int LANES>
void launch32_shape(const sph_compressible_params* p, const sph_compressible_state* st, const float4* r0,
                    const float4* r1, double* a, double* b, double* c, float4* n0, float4* n1, cudaStream_t s) {
    const int64_t n = p->dom.n;
    const Plan32 v = plan_view(st, DIM, n);
    k_comp32<DIM, UPDATE, LANES><<<grid_for(n * LANES, 128), 128, 0, s>>>(
        r0, r1, v.ga, v.gb, st->row_ptr, n, st->plan_width, (float)p->gamma, (float)p->eta, p->dt, a, b, c, n0, n1);
}

template <int DIM, bool UPDATE>
void launch32_dim(int lanes, const sph_compressible_params* p, const sph_compressible_state* st, const float4* r0,
                  const float4* r1, double* a, double* b, double* c, float4* n0, float4* n1, cudaStream_t s) {
    switch (lanes) {
        case 2: launch32_shape<DIM, UPDATE, 2>(p, st, r0, r1, a, b, c, n0, n1, s); break;
        case 4: launch32_shape<DIM, UPDATE, 4>(p, st, r0, r1, a, b, c, n0, n1, s); break;
        case 8: launch32_shape<DIM, UPDATE, 8>(p, st, r0, r1, a, b, c, n0, n1, s); break;
        default: launch32_shape<DIM, UPDATE, 1>(p, st, r0, r1, a, b, c, n0, n1, s); break;
    }
}

template <bool UPDATE>
void launch32(int lanes, const sph_compressible_params* p, const sph_compressible_state* st, const float4* r0,
              const float4* r1, double* a, double* b, double* c, float4* n0, float4* n1, cudaStream_t s) {
    if (p->dom.dim == 2)
        launch32_dim<2, UPDATE>(lanes, p, st, r0, r1, a, b, c, n0, n1, s);
    else
        launch32_dim<3, UPDATE>(lanes, p, st, r0, r1, a, b, c, n0, n1, s);
}

}  // namespace

extern "C" int sph_compressible_plan_bytes(sph_ctx* ctx, const sph_compressible_params* p,
                                           const sph_compressible_state* st, int64_t* bytes_host, void* stream) {
    if (!ctx || !bytes_host) return SPH_ERR_ARG;
    int r = check(p, st);
    if (r) return r;
    int64_t n = p->dom.n, nnz = 0, maxrow = 0;
    if (n > 0) {
        r = sph_row_stats(ctx, st->row_ptr, n, as_stream(stream), &nnz, &maxrow);
        if (r) return r;
    }
    *bytes_host = (int64_t)plan_bytes_for(p->dom.dim, n, maxrow);
    return SPH_OK;
}

extern "C" int sph_compressible_plan(sph_ctx* ctx, const sph_compressible_params* p, sph_compressible_state* st,
                                     void* stream) {
    if (!ctx) return SPH_ERR_ARG;
    int r = check(p, st);
    if (r) return r;
    st->plan_width = 0;
    const int64_t n = p->dom.n;
    if (n == 0) return SPH_OK;
    if (!st->plan || ((uintptr_t)st->plan & 15u)) return SPH_ERR_ARG;
    cudaStream_t s = as_stream(stream);
    int64_t nnz = 0, maxrow = 0;
    r = sph_row_stats(ctx, st->row_ptr, n, s, &nnz, &maxrow);
    if (r) return r;
    if (maxrow > (1 << 20)) return SPH_ERR_LIMIT;
    if (st->plan_bytes < (int64_t)plan_bytes_for(p->dom.dim, n, maxrow)) return SPH_ERR_CAPACITY;
    const int width = maxrow > 0 ? (int)maxrow : 1;
    float4* ga = reinterpret_cast<float4*>(st->plan);
    void* gb = reinterpret_cast<unsigned char*>(st->plan) + plan_entries(n, width) * 16;
    const CompK K = consts(p);
    if (p->dom.dim == 2)
        k_comp_geo<2><<<grid_for(n, 128), 128, 0, s>>>(st->pos, st->vol, st->B, st->row_ptr, st->col, n, K, width,
                                                       ga, gb);
    else
        k_comp_geo<3><<<grid_for(n, 128), 128, 0, s>>>(st->pos, st->vol, st->B, st->row_ptr, st->col, n, K, width,
                                                       ga, gb);
    SPH_LAUNCH_CHECK(ctx);
    SPH_CUDA(ctx, cudaStreamSynchronize(s));
    st->plan_width = width;
    return SPH_OK;
}

extern "C" int sph_compressible_rates(sph_ctx* ctx, const sph_compressible_params* p,
                                      const sph_compressible_state* st, double* drho, double* dmom, double* dE,
                                      void* stream) {
    if (!ctx) return SPH_ERR_ARG;
    int r = check(p, st);
    if (r) return r;
    if (p->dom.n == 0) return SPH_OK;
    if (!drho || !dmom || !dE) return SPH_ERR_ARG;
    r = check_plan(p, st);
    if (r) return r;
    cudaStream_t s = as_stream(stream);
    const int64_t n = p->dom.n;
    if (p->precision == SPH_FP64) {
        launch_rates(p, st, consts(p), drho, dmom, dE, s);
    } else {
        float4* rec = (float4*)sph_scratch(ctx, S_MISC2, (size_t)n * 32, &r);
        if (r) return r;
        launch_rec(p, st, rec, rec + n, s);
        launch32<false>(ctx->lanes[SPH_PASS_COMPRESSIBLE], p, st, rec, rec + n, drho, dmom, dE, nullptr, nullptr, s);
    }
    SPH_LAUNCH_CHECK(ctx);
    return SPH_OK;
}

extern "C" int sph_compressible_step(sph_ctx* ctx, const sph_compressible_params* p,
                                     const sph_compressible_state* st, int nsteps, void* stream) {
    if (!ctx || nsteps < 0) return SPH_ERR_ARG;
    int r = check(p, st);
    if (r) return r;
    const int64_t n = p->dom.n;
    if (n == 0 || nsteps == 0) return SPH_OK;
    r = check_plan(p, st);
    if (r) return r;
    const int dim = p->dom.dim;
    cudaStream_t s = as_stream(stream);
    if (p->precision == SPH_FP32_KAHAN) {
        // double-buffered records: step k reads buffer k % 2 and writes the other
        float4* a = (float4*)sph_scratch(ctx, S_MISC2, (size_t)n * 32, &r);
        if (r) return r;
        float4* b = (float4*)sph_scratch(ctx, S_MISC3, (size_t)n * 32, &r);
        if (r) return r;
        launch_rec(p, st, a, a + n, s);
        const int lanes = ctx->lanes[SPH_PASS_COMPRESSIBLE];
        for (int k = 0; k < nsteps; ++k) {
            launch32<true>(lanes, p, st, a, a + n, st->rho, st->mom, st->E, b, b + n, s);
            SPH_LAUNCH_CHECK(ctx);
            float4* t = a;
            a = b;
            b = t;
        }
        return SPH_OK;
    }
    double* rates = (double*)sph_scratch(ctx, S_MISC2, (size_t)n * (dim + 2) * 8, &r);
    if (r) return r;
    double *drho = rates, *dmom = rates + n, *dE = rates + (int64_t)(dim + 1) * n;
    const CompK K = consts(p);
    for (int k = 0; k < nsteps; ++k) {
        launch_rates(p, st, K, drho, dmom, dE, s);
        k_comp_update<<<grid_for(n, 256), 256, 0, s>>>(st->rho, st->mom, st->E, drho, dmom, dE, n, dim, p->dt);
        SPH_LAUNCH_CHECK(ctx);
    }
    return SPH_OK;
}
