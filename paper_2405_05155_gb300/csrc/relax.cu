// a10/a11: Laguerre-Gauss particle relaxation (Sec. 2.3.2; Eqs. 7-8) and its
// residual.  Positions move every step, so the neighbour sets change.
//  - float32 step (default): a buffered neighbour list of cut-off 2h + skin,
//    rebuilt only when twice the largest displacement since its build exceeds the
//    skin; every step decides each listed pair at 2h exactly, accumulates the
//    acceleration with a block-level max of |a|, and a pointwise update follows
//    (dt = 0.25 sqrt(h/max|a|), x += a dt^2/2, projection back inside the body).
//  - float32 step with skin 0, and the single acceleration evaluation: no list; one
//    sweep over the neighbouring cells screens every candidate (the a2 screen and
//    float64 band, so the pair set equals the list builder's) and accumulates.
//  - float64 step: explicit CSR lists (count, scan, fill) every step, launched back
//    to back without host synchronisation.
// In both list forms a device flag records a capacity overflow (or a stale list),
// after which the remaining steps are no-ops and the host regrows (or rebuilds) the
// list and resumes from that step.
#include <algorithm>
#include <mutex>
#include <set>

#include "common.cuh"
#include "neighbors.cuh"

namespace {

struct Spheres {
    int count;
    double c[SPH_MAX_SPHERES][3];
    double r[SPH_MAX_SPHERES];
    float ch[SPH_MAX_SPHERES][3], cl[SPH_MAX_SPHERES][3], rf[SPH_MAX_SPHERES];
};

struct RelaxK {
    double h, dp, scale;           // scale = 2 p0 / rho
    double gcoef;                  // gs coefficient of the relaxation kernel (h^-(d+2) included)
    double gcoef_lg;               // LG gs coefficient -ahat h^-(d+2) / 3 (residual)
    double gcoef_tw;               // Wendland gs coefficient -5 alpha h^-(d+2) (residual)
    double inv_h;
    double rc2_tw;                 // (1.6 h)^2 for the truncated residual
    double surf_coef;              // 3D Laguerre-Gauss closed form: 2 pi ahat / h
    double rc;                     // cut-off of the relaxation kernel, kappa h
    double w_norm;                 // alpha_d h^-d of the relaxation kernel
    int kernel;                    // SPH_LAGUERRE_GAUSS or SPH_WENDLAND_C2
    float gcoef_f, inv_h_f, inv_h2_f, scale_f, surf_coef_f, h_f, dp_f;
};

// Gauss-Legendre rule of the surface integrals that have no closed form (nodes on
// [0, 1] and their weights), set once per device from the host.
constexpr int kGL = 48;
__constant__ double c_gl_u[kGL], c_gl_w[kGL];

// Shape of the relaxation kernel, W / (alpha_d h^-d), uncut.
__device__ __forceinline__ double kernel_shape(int kernel, double q) {
    if (kernel == SPH_WENDLAND_C2) {
        double t = 1.0 - 0.5 * q;
        return t * t * t * t * (2.0 * q + 1.0);
    }
    double q2 = q * q;
    return (1.0 - 0.5 * q2 + q2 * q2 / 6.0) * exp(-q2);
}

// Signed distance to the union of spheres (circles in 2D) and its unit normal
// (first minimiser).
template <int DIM = 3>
__device__ __forceinline__ double sdf64(const Spheres& S, const double* x, double* g) {
    double best = 0.0;
    int arg = 0;
    for (int k = 0; k < S.count; ++k) {
        double d2 = 0.0;
        for (int a = 0; a < DIM; ++a) {
            double dx = x[a] - S.c[k][a];
            d2 += dx * dx;
        }
        double d = sqrt(d2) - S.r[k];
        if (k == 0 || d < best) { best = d; arg = k; }
    }
    double rr[3] = {0.0, 0.0, 0.0}, nr2 = 0.0;
    for (int a = 0; a < DIM; ++a) {
        rr[a] = x[a] - S.c[arg][a];
        nr2 += rr[a] * rr[a];
    }
    double nr = sqrt(nr2);
    for (int a = 0; a < DIM; ++a) g[a] = nr > 0.0 ? rr[a] / nr : (a == 0 ? 1.0 : 0.0);
    return best;
}

// Same in float32 from a hi+lo position (differences keep float32 accuracy).
__device__ __forceinline__ float sdf32(const Spheres& S, const float* xh, const float* xl, float* g) {
    float best = 0.0f;
    int arg = 0;
    float brx = 0.f, bry = 0.f, brz = 0.f;
    for (int k = 0; k < S.count; ++k) {
        float dx = (xh[0] - S.ch[k][0]) + (xl[0] - S.cl[k][0]);
        float dy = (xh[1] - S.ch[k][1]) + (xl[1] - S.cl[k][1]);
        float dz = (xh[2] - S.ch[k][2]) + (xl[2] - S.cl[k][2]);
        float d = sqrtf(dx * dx + dy * dy + dz * dz) - S.rf[k];
        if (k == 0 || d < best) { best = d; arg = k; brx = dx; bry = dy; brz = dz; }
    }
    float nr = sqrtf(brx * brx + bry * bry + brz * brz);
    if (nr > 0.0f) { float in = 1.0f / nr; g[0] = brx * in; g[1] = bry * in; g[2] = brz * in; }
    else { g[0] = 1.0f; g[1] = 0.0f; g[2] = 0.0f; }
    (void)arg;
    return best;
}

// Half-space surface integral I(d) = 2 pi int_d^{2h} z (W(z) - W(2h)) dz of the 3D
// Laguerre-Gauss kernel: with t = z/h the antiderivative of t w(t) is
// -(1/12) e^{-t^2} (5 - t^2 + t^4), and W(2h) = ahat h^-3 (5/3) e^{-4}.
template <typename R>
__device__ __forceinline__ R surface_lg(R d, R inv_h, R coef) {   // coef = 2 pi ahat / h
    R t = d * inv_h;
    t = t < R(0) ? R(0) : (t > R(2) ? R(2) : t);
    R t2 = t * t;
    const R e4 = R(0.018315638888734179);          // e^-4
    R prim2 = -(R(1) / R(12)) * e4 * R(17);        // at t = 2: 5 - 4 + 16 = 17
    R primt = -(R(1) / R(12)) * exp(-t2) * (R(5) - t2 + t2 * t2);
    R wcut = (R(5) / R(3)) * e4;
    return coef * ((prim2 - primt) - R(0.5) * wcut * (R(4) - t2));
}

__device__ __forceinline__ void atomic_max_nonneg(unsigned* addr, float v) {
    atomicMax(addr, __float_as_uint(v));
}

// ---------------------------------------------------------------- acceleration
// Surface term I(d) of the relaxation kernel (the integral of -dW/dr z/|r| over the
// support beyond the tangent line or plane at distance d): the closed form for the
// 3D Laguerre-Gauss kernel, else
//   2D: 2 int_0^Y (W(sqrt(d^2 + y^2)) - W(kappa h)) dy,  Y = sqrt((kappa h)^2 - d^2),
//   3D: 2 pi int_d^{kappa h} z (W(z) - W(kappa h)) dz,
// by the Gauss-Legendre rule in constant memory.
template <int DIM>
__device__ double surface_term(double d, const RelaxK& K) {
    d = fmin(fmax(d, 0.0), K.rc);
    if (DIM == 3 && K.kernel == SPH_LAGUERRE_GAUSS) return surface_lg<double>(d, K.inv_h, K.surf_coef);
    const double wcut = kernel_shape(K.kernel, K.rc * K.inv_h);
    double acc = 0.0;
    if (DIM == 2) {
        const double Y = sqrt(fmax(K.rc * K.rc - d * d, 0.0));
        for (int k = 0; k < kGL; ++k) {
            const double y = Y * c_gl_u[k];
            acc += c_gl_w[k] * (kernel_shape(K.kernel, sqrt(d * d + y * y) * K.inv_h) - wcut);
        }
        return 2.0 * Y * K.w_norm * acc;
    }
    for (int k = 0; k < kGL; ++k) {
        const double z = d + (K.rc - d) * c_gl_u[k];
        acc += c_gl_w[k] * z * (kernel_shape(K.kernel, z * K.inv_h) - wcut);
    }
    return 2.0 * SPH_PI * (K.rc - d) * K.w_norm * acc;
}

template <int DIM>
__device__ __forceinline__ double relax_gs(double q, const RelaxK& K) {
    return K.kernel == SPH_WENDLAND_C2 ? wendland_gs<double>(q, K.gcoef) : lg_gs<double>(q, K.gcoef);
}

template <int DIM>
__global__ void k_relax_acc64(const double* __restrict__ pos, const double* __restrict__ vol, int64_t n,
                              const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col, Spheres S,
                              RelaxK K, double* __restrict__ acc, unsigned* __restrict__ amax,
                              const int* __restrict__ flags) {
    __shared__ unsigned smax;
    if (threadIdx.x == 0) smax = 0u;
    __syncthreads();
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    bool skip = flags[FLAG_CAPACITY] != 0;
    if (i < n && !skip) {
        double xi[DIM];
        for (int a = 0; a < DIM; ++a) xi[a] = pos[a * n + i];
        double s[DIM];
        for (int a = 0; a < DIM; ++a) s[a] = 0.0;
        for (int64_t p = row_ptr[i], e = row_ptr[i + 1]; p < e; ++p) {
            int j = col[p];
            double r[DIM], d2 = 0.0;
            for (int a = 0; a < DIM; ++a) { r[a] = xi[a] - pos[a * n + j]; d2 += r[a] * r[a]; }
            double gs = relax_gs<DIM>(sqrt(d2) * K.inv_h, K) * vol[j];
            for (int a = 0; a < DIM; ++a) s[a] += gs * r[a];
        }
        double g[DIM];
        double phi = sdf64<DIM>(S, xi, g);
        double I = surface_term<DIM>(phi < 0.0 ? -phi : 0.0, K);
        double m2 = 0.0;
        for (int c = 0; c < DIM; ++c) {
            double a = -K.scale * (s[c] + I * g[c]);
            m2 += a * a;
            acc[c * n + i] = a;
        }
        atomic_max_nonneg(&smax, __double2float_ru(sqrt(m2)));
    }
    __syncthreads();
    if (threadIdx.x == 0 && smax) atomicMax(amax, smax);
}

// exact float64 max of |a| (the float32 block max above only bounds it; a second
// pass takes the exact value among candidates >= the bound's float32 lower edge)
template <int DIM>
__global__ void k_amax64_exact(const double* __restrict__ acc, int64_t n, const unsigned* __restrict__ amax_f,
                               unsigned long long* __restrict__ amax_d, const int* __restrict__ flags) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || flags[FLAG_CAPACITY]) return;
    double m2 = 0.0;
    for (int a = 0; a < DIM; ++a) m2 += acc[a * n + i] * acc[a * n + i];
    double m = sqrt(m2);
    float bound = __uint_as_float(*amax_f);
    if (__double2float_ru(m) == bound) atomicMax(amax_d, (unsigned long long)__double_as_longlong(m));
}

// pos[a][i] = xh + xl of slot m (i = sorted[m]): the positions back to the
// caller's order, in float64.
__global__ void k_relax_scatter_pos(const float4* __restrict__ rec, const int32_t* __restrict__ sorted, int64_t n,
                                    double* __restrict__ pos) {
    int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= n) return;
    int i = sorted[m];
    float4 a = rec[2 * m], b = rec[2 * m + 1];
    pos[i] = (double)a.x + (double)b.x;
    pos[n + i] = (double)a.y + (double)b.y;
    pos[2 * n + i] = (double)a.z + (double)b.z;
}

// x + d for a float-float x = xh + xl and a float32 d: the sum xh + d and its
// rounding error (Knuth's TwoSum), the error added to xl, and the pair
// renormalised by a second TwoSum.  Every operation rounds on its own.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    float bv = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bv)), __fsub_rn(b, bv));
}

__device__ __forceinline__ void ff_add(float& xh, float& xl, float d) {
    float s, e, h, l;
    two_sum(xh, d, s, e);
    two_sum(s, __fadd_rn(xl, e), h, l);
    xh = h;
    xl = l;
}

// The float64 neighbour predicate (unfused sum of squares, as the list builder's)
// for the float-float positions xi and those of record r.
__device__ __forceinline__ bool within_ff(const double* xi, const F8& r, double rc2) {
    double d2 = 0.0;
    for (int a = 0; a < 3; ++a) {
        double dx = __dsub_rn(xi[a], (double)r.v[a] + (double)r.v[4 + a]);
        double sq = __dmul_rn(dx, dx);
        d2 = a == 0 ? sq : __dadd_rn(d2, sq);
    }
    return d2 <= rc2;
}

// ---------------------------------------------------------------- update
template <int DIM>
__global__ void k_relax_update64(double* __restrict__ pos, int64_t n, const double* __restrict__ acc,
                                 const unsigned long long* __restrict__ amax_d, Spheres S, RelaxK K,
                                 const int* __restrict__ flags) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || flags[FLAG_CAPACITY]) return;
    double am = __longlong_as_double((long long)*amax_d);
    double x[DIM];
    for (int c = 0; c < DIM; ++c) x[c] = pos[c * n + i];
    if (am > 0.0) {
        double dt = 0.25 * sqrt(K.h / am);
        for (int c = 0; c < DIM; ++c) x[c] = x[c] + 0.5 * acc[c * n + i] * (dt * dt);
    }
    double g[DIM];
    double phi = sdf64<DIM>(S, x, g);
    if (phi > -0.5 * K.dp) {
        double sh = phi + 0.5 * K.dp;
        for (int c = 0; c < DIM; ++c) x[c] = x[c] - sh * g[c];
    }
    for (int c = 0; c < DIM; ++c) pos[c * n + i] = x[c];
}

__global__ void k_relax_update32(double* __restrict__ pos, int64_t n, const float4* __restrict__ acc,
                                 const unsigned* __restrict__ amax, Spheres S, RelaxK K,
                                 const int* __restrict__ flags) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || flags[FLAG_CAPACITY]) return;
    float am = __uint_as_float(*amax);
    double x[3] = {pos[i], pos[n + i], pos[2 * n + i]};
    if (am > 0.0f) {
        float sc = (K.h_f * 0.03125f) / am;         // a dt^2/2 = a (h/32)/max|a|
        float4 a = acc[i];
        x[0] += (double)(a.x * sc);
        x[1] += (double)(a.y * sc);
        x[2] += (double)(a.z * sc);
    }
    float xh[3], xl[3], g[3];
    for (int c = 0; c < 3; ++c) { xh[c] = (float)x[c]; xl[c] = (float)(x[c] - (double)xh[c]); }
    float phi = sdf32(S, xh, xl, g);
    if (phi > -0.5f * K.dp_f) {
        float sh = phi + 0.5f * K.dp_f;
        for (int c = 0; c < 3; ++c) x[c] -= (double)(sh * g[c]);
    }
    for (int c = 0; c < 3; ++c) pos[c * n + i] = x[c];
}

// ---------------------------------------------------------------- residual
template <int DIM>
__global__ void k_relax_residual(const double* __restrict__ pos, const double* __restrict__ vol, int64_t n,
                                 const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col, Spheres S,
                                 RelaxK K, double* __restrict__ partial) {
    __shared__ double sh[3][256];
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double e_lg = 0.0, e_tw = 0.0, cnt = 0.0;
    if (i < n) {
        double xi[DIM];
        for (int a = 0; a < DIM; ++a) xi[a] = pos[a * n + i];
        double g[DIM];
        double phi = sdf64<DIM>(S, xi, g);
        if (phi < -2.0 * K.h) {
            double s1[DIM], s2[DIM];
            for (int a = 0; a < DIM; ++a) s1[a] = s2[a] = 0.0;
            for (int64_t p = row_ptr[i], e = row_ptr[i + 1]; p < e; ++p) {
                int j = col[p];
                double r[DIM], d2 = 0.0, d2u = 0.0;
                for (int a = 0; a < DIM; ++a) {
                    r[a] = xi[a] - pos[a * n + j];
                    d2 += r[a] * r[a];
                    double sq = __dmul_rn(r[a], r[a]);
                    d2u = a == 0 ? sq : __dadd_rn(d2u, sq);
                }
                double q = sqrt(d2) * K.inv_h;
                double w = vol[j];
                double g1 = lg_gs<double>(q, K.gcoef_lg) * w;
                double g2 = d2u <= K.rc2_tw ? wendland_gs<double>(q, K.gcoef_tw) * w : 0.0;
                for (int a = 0; a < DIM; ++a) { s1[a] += g1 * r[a]; s2[a] += g2 * r[a]; }
            }
            double h2 = K.h * K.h, m1 = 0.0, m2 = 0.0;
            for (int a = 0; a < DIM; ++a) { m1 += s1[a] * s1[a]; m2 += s2[a] * s2[a]; }
            e_lg = h2 * m1;
            e_tw = h2 * m2;
            cnt = 1.0;
        }
    }
    sh[0][threadIdx.x] = e_lg;
    sh[1][threadIdx.x] = e_tw;
    sh[2][threadIdx.x] = cnt;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o)
            for (int c = 0; c < 3; ++c) sh[c][threadIdx.x] += sh[c][threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int c = 0; c < 3; ++c) partial[3 * blockIdx.x + c] = sh[c][0];
}

__global__ void k_sum_partials(const double* __restrict__ partial, int nb, double* __restrict__ out) {
    __shared__ double sh[3][256];
    double a[3] = {0, 0, 0};
    for (int b = threadIdx.x; b < nb; b += blockDim.x)
        for (int c = 0; c < 3; ++c) a[c] += partial[3 * b + c];
    for (int c = 0; c < 3; ++c) sh[c][threadIdx.x] = a[c];
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o)
            for (int c = 0; c < 3; ++c) sh[c][threadIdx.x] += sh[c][threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int c = 0; c < 3; ++c) out[c] = sh[c][0];
}

// ---------------------------------------------------------------- float32 cell sweep
// The float32 pair loops screen candidates with the float32 position copy of a
// cell sort (the a2 screen, with the float64 decision inside the rounding band,
// so the pair set is the list builder's).  Threads walk the particles in cell
// order, so the candidates of neighbouring threads are the same cells (L1 reuse).

// (x - float(x), V) per particle in sorted order: the float32 low parts of the position
__global__ void k_relax_pack_lo(const double* __restrict__ pos, const double* __restrict__ vol, int64_t n,
                                const int32_t* __restrict__ sorted, const float4* __restrict__ p32,
                                float4* __restrict__ lo) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    int j = sorted[k];
    float4 h = p32[k];
    lo[k] = make_float4((float)(pos[j] - (double)h.x), (float)(pos[n + j] - (double)h.y),
                        (float)(pos[2 * n + j] - (double)h.z), (float)vol[j]);
}

template <int N>
__device__ __forceinline__ float pick(const float (&a)[N], int k) {
    float v = a[0];
#pragma unroll
    for (int t = 1; t < N; ++t) v = k == t ? a[t] : v;
    return v;
}

// Visits, in cell order, the sorted slots of the cells within R of the particle's
// cell ci (cells of edge >= rc / R) whose box lies within sqrt(thr) of xh.  The
// outermost cells extend to infinity outwards (clamped particles outside the box
// lie in them).  Along x the passing cells of a row are consecutive (the distance
// to the slabs falls, then rises), so a row is one run of sorted slots.
template <int R, typename F>
__device__ __forceinline__ void sweep_cells(const float* xh, const int* ci, const CellGrid& g,
                                            const int32_t* __restrict__ start, float thr, F&& visit) {
    constexpr int W = 2 * R + 1;
    float sd[3][W];   // squared distance to the cell slabs ci + d, d in [-R, R], per axis
    int dlo[3], dhi[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        dlo[a] = max(ci[a] - R, 0) - ci[a];
        dhi[a] = min(ci[a] + R, g.n[a] - 1) - ci[a];
#pragma unroll
        for (int d = -R; d <= R; ++d) {
            int c = ci[a] + d;
            float x = xh[a];
            float b0 = (float)(g.lo[a] + c * g.size[a]), b1 = (float)(g.lo[a] + (c + 1) * g.size[a]);
            float gap = 0.0f;
            if (c > 0 && x < b0) gap = b0 - x;
            if (c < g.n[a] - 1 && x > b1) gap = x - b1;
            sd[a][d + R] = gap * gap;
        }
    }
#pragma unroll 1
    for (int dz = dlo[2]; dz <= dhi[2]; ++dz) {
        const float sz = pick<W>(sd[2], dz + R);
#pragma unroll 1
        for (int dy = dlo[1]; dy <= dhi[1]; ++dy) {
            const float syz = sz + pick<W>(sd[1], dy + R);
            if (syz > thr) continue;
            int a = W, b = -1;
#pragma unroll
            for (int d = 0; d < W; ++d) {
                bool ok = d - R >= dlo[0] && d - R <= dhi[0] && syz + sd[0][d] <= thr;
                if (ok && a == W) a = d;
                if (ok) b = d;
            }
            if (b < 0) continue;
            int row = ((ci[2] + dz) * g.n[1] + ci[1] + dy) * g.n[0] + ci[0] - R;
            int e = start[row + b + 1];
            for (int m = start[row + a]; m < e; ++m) visit(m);
        }
    }
}

// Compensated sum of the pair terms: (x, y) on the paired float32 instructions,
// z on its own; the same Kahan steps on every component.
struct LgSum {
    Kahan2 xy;
    Kahan<float> z;
    __device__ __forceinline__ void init() { xy.init(); z.init(); }
    __device__ __forceinline__ void value(float* out) const {
        float2 v = xy.value();
        out[0] = v.x;
        out[1] = v.y;
        out[2] = z.value();
    }
};

// Pair term of Eq. 7 for an accepted pair: r = x_i - x_j from the high parts'
// difference (dx, dy, dz) and the low parts; grad W^LG_ij V_j = gs r with gs a
// function of q^2 = r^2/h^2 alone (Eq. 8 divided by r), so no square root.
__device__ __forceinline__ void lg_pair(LgSum& s, float dx, float dy, float dz, const float* xl, float4 q,
                                        const RelaxK& K) {
    const float2 lxy = __ffma2_rn(make_float2(q.x, q.y), make_float2(-1.0f, -1.0f), make_float2(xl[0], xl[1]));
    const float2 rxy = __fadd2_rn(make_float2(dx, dy), lxy);
    const float rz = __fadd_rn(dz, __fsub_rn(xl[2], q.z));
    const float d2 = fmaf(rz, rz, fmaf(rxy.y, rxy.y, rxy.x * rxy.x));
    const float q2 = d2 * K.inv_h2_f;
    const float gs = K.gcoef_f * expf(-q2) * fmaf(q2, q2 - 5.0f, 9.0f) * q.w;
    s.xy.add(__fmul2_rn(make_float2(gs, gs), rxy));
    s.z.add(gs * rz);
}

// Acceleration of Eq. 8 from the pair sum and the surface term; returns |a|.
__device__ __forceinline__ float lg_finish(const Spheres& S, const RelaxK& K, const float* xh, const float* xl,
                                           const float* sum, float4* out) {
    float g3[3];
    float phi = sdf32(S, xh, xl, g3);
    float I = surface_lg<float>(phi < 0.0f ? -phi : 0.0f, K.inv_h_f, K.surf_coef_f);
    float a0 = -K.scale_f * (sum[0] + I * g3[0]);
    float a1 = -K.scale_f * (sum[1] + I * g3[1]);
    float a2 = -K.scale_f * (sum[2] + I * g3[2]);
    *out = make_float4(a0, a1, a2, 0.0f);
    return sqrtf(a0 * a0 + a1 * a1 + a2 * a2);
}

// One sweep over the cells of edge h within two of the particle's screens every
// candidate and accumulates the Laguerre-Gauss gradient of the accepted pairs
// at once (no list): the single-evaluation form and the skin-0 step.
template <int R>
__global__ void __launch_bounds__(256) k_relax_acc_cells(const float4* __restrict__ p32, const float4* __restrict__ lo,
                                                        const int32_t* __restrict__ start, CellGrid g,
                                                        const unsigned* __restrict__ absmax, double rc2,
                                                        const double* __restrict__ pos, int64_t n, Spheres S,
                                                        RelaxK K, float4* __restrict__ acc,
                                                        unsigned* __restrict__ amax) {
    __shared__ unsigned smax;
    if (threadIdx.x == 0) smax = 0u;
    __syncthreads();
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) {
        float4 me = p32[k];
        float4 ml = lo[k];
        int i = __float_as_int(me.w);
        float xh[3] = {me.x, me.y, me.z}, xl[3] = {ml.x, ml.y, ml.z};
        double xi[3] = {pos[i], pos[n + i], pos[2 * n + i]};
        int ci[3];
        for (int a = 0; a < 3; ++a) ci[a] = nb::cell_coord(xi[a], a, g);
        nb::Band band = nb::make_band(absmax, 0.0, rc2, 3);
        LgSum s;
        s.init();
        sweep_cells<R>(xh, ci, g, start, band.hi * 1.0001f, [&](int m) {
            float4 p = p32[m];
            int j = __float_as_int(p.w);
            if (j == i) return;
            float dx = xh[0] - p.x, dy = xh[1] - p.y, dz = xh[2] - p.z;
            float d2s = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
            if (d2s > band.hi) return;
            if (d2s >= band.lo && !nb::exact_within(pos, n, 3, xi, j, g, rc2)) return;
            lg_pair(s, dx, dy, dz, xl, lo[m], K);
        });
        float sum[3];
        s.value(sum);
        atomic_max_nonneg(&smax, lg_finish(S, K, xh, xl, sum, &acc[i]));
    }
    __syncthreads();
    if (threadIdx.x == 0 && smax) atomicMax(amax, smax);
}

// ---------------------------------------------------------------- float32 skin lists
// Positions move by at most h/32 per step, and after the first steps of a run the
// largest net displacement grows slowly.  The float32 step therefore keeps a list
// of cut-off 2h + skin (a buffered, Verlet-style list) and rebuilds it only when
// two particles could have come within 2h unlisted: when twice the largest
// displacement since the build exceeds the skin.  Every step still decides each
// listed pair at 2h exactly (float32 screen, float64 inside the rounding band), so
// the pair set is the one a fresh list gives.
//
// Everything runs in the cell order of the last build ("slots"): the list holds
// slots; the current positions are kept per slot in one 32-byte record (rec[2m]:
// float32 high parts and the particle index bits; rec[2m+1]: low parts and V), so
// that a gathered neighbour costs one sector; the build's copies (p32, lo) are the
// reference for the displacement.  While the list lives the position is that
// pair, x = xh + xl (a float-float number: ~48 significant bits), updated with
// float32 operations (GB300's float64 pipe is slow); float64 appears only in the
// exact decisions inside the rounding band, and x is written back to the caller's
// float64 array before a rebuild and at the end of the call.  The list is sliced by 32 slots (entry k of slot
// m at (m / 32) * cap * 32 + k * 32 + m % 32), so a warp reads 128 contiguous bytes
// per entry.
//
// Control words (ctl, float bits as unsigned): [0..1] max |a| of the steps of even
// and odd index, [2..3] the largest displacement since the build, read by the step
// of that parity, [4] the longest row found by a build that overflowed the list.
// Each kernel clears the word of the other parity that the next kernel fills, so a
// step needs no memset; a build clears them all.
constexpr int kCtlAmax = 0, kCtlDisp = 2, kCtlNeed = 4;

template <int R>
__global__ void __launch_bounds__(256) k_relax_skin_build(const float4* __restrict__ p32, const float4* __restrict__ lo,
                                                         const int32_t* __restrict__ start, CellGrid g,
                                                         const unsigned* __restrict__ absmax, double rb2,
                                                         const double* __restrict__ pos, int64_t n, int cap,
                                                         int32_t* __restrict__ col, int32_t* __restrict__ rowlen,
                                                         float4* __restrict__ rec, unsigned* __restrict__ ctl, int step,
                                                         int* __restrict__ flags) {
    int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= n) return;
    float4 me = p32[m];
    rec[2 * m] = me;
    rec[2 * m + 1] = lo[m];
    int i = __float_as_int(me.w);
    float xh[3] = {me.x, me.y, me.z};
    int ci[3];
    for (int a = 0; a < 3; ++a) ci[a] = nb::cell_coord(pos[a * n + i], a, g);
    // superset of the pairs within 2h + skin: the float32 screen's upper edge
    nb::Band band = nb::make_band(absmax, 0.0, rb2, 3);
    int32_t* out = col + (m >> 5) * (int64_t)cap * 32 + (m & 31);
    int len = 0;
    sweep_cells<R>(xh, ci, g, start, band.hi * 1.0001f, [&](int q) {
        if (q == (int)m) return;
        float4 p = p32[q];
        float dx = xh[0] - p.x, dy = xh[1] - p.y, dz = xh[2] - p.z;
        float d2s = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
        if (d2s > band.hi) return;
        if (len < cap) out[(int64_t)len * 32] = q;
        ++len;
    });
    rowlen[m] = len;
    if (len > cap) {
        atomicMax(&ctl[kCtlNeed], (unsigned)len);
        atomicCAS(&flags[FLAG_CAPACITY], 0, step + 1);
    }
}

__device__ __forceinline__ bool relax_halted(const int* flags) {
    return (flags[FLAG_BAD_INPUT] | flags[FLAG_CAPACITY] | flags[FLAG_STALE]) != 0;
}

// Step `step`: the acceleration from the list, LANES lanes per slot.  Skips the
// step (and flags it) when the list is stale, so that every later launch of the
// batch is a no-op and the host resumes from this step after a rebuild.
constexpr int kWalkChunk = 8;

template <int LANES>
__global__ void __launch_bounds__(256, 4) k_relax_walk(const float4* __restrict__ rec,
                                                   const int32_t* __restrict__ col, const int32_t* __restrict__ rowlen,
                                                   int cap, int64_t n,
                                                   const unsigned* __restrict__ absmax, double lmax, double rc2,
                                                   float skin, Spheres S, RelaxK K,
                                                   float4* __restrict__ acc, unsigned* __restrict__ ctl, int step,
                                                   int* __restrict__ flags) {
    __shared__ unsigned smax;
    __shared__ int skip;
    if (threadIdx.x == 0) {
        smax = 0u;
        bool halted = relax_halted(flags);
        float d = __uint_as_float(ctl[kCtlDisp + (step & 1)]);
        bool stale = !(2.0f * d <= skin);     // also on a non-finite displacement
        if (!halted && stale) atomicCAS(&flags[FLAG_STALE], 0, step + 1);
        skip = halted || stale;
        if (!skip && blockIdx.x == 0) ctl[kCtlDisp + ((step + 1) & 1)] = 0u;
    }
    __syncthreads();
    if (skip) return;
    int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t m = gt / LANES;
    int lane = (int)(gt % LANES);
    bool live = m < n;
    int64_t mm = live ? m : 0;
    const F8 own = ldg8((const float*)&rec[2 * mm]);
    float xh[3] = {own.v[0], own.v[1], own.v[2]}, xl[3] = {own.v[4], own.v[5], own.v[6]};
    double xi[3];
    for (int a = 0; a < 3; ++a) xi[a] = (double)xh[a] + (double)xl[a];
    // positions may have moved by skin/2 since the build's |x| maximum
    nb::Band band = nb::make_band(absmax, lmax, rc2, 3);
    const int32_t* rowc = col + (mm >> 5) * (int64_t)cap * 32 + (mm & 31);
    int len = live ? rowlen[mm] : 0;
    LgSum s;
    s.init();
    // the list entries are read kWalkChunk at a time, the next chunk's loads in
    // flight while this chunk's records are gathered and summed
    int qa[kWalkChunk], qb[kWalkChunk];
    auto fetch = [&](int k0, int* q) {
#pragma unroll
        for (int u = 0; u < kWalkChunk; ++u) {
            int k = k0 + u * LANES;
            q[u] = k < len ? ldg1_stream(&rowc[(int64_t)k * 32]) : -1;
        }
    };
    fetch(lane, qa);
    for (int k0 = lane; k0 < len; k0 += kWalkChunk * LANES) {
        fetch(k0 + kWalkChunk * LANES, qb);
#pragma unroll
        for (int u = 0; u < kWalkChunk; ++u) {
            const int q = qa[u];
            if (q < 0) break;
            const F8 r = ldg8((const float*)&rec[2 * q]);
            float dx = xh[0] - r.v[0], dy = xh[1] - r.v[1], dz = xh[2] - r.v[2];
            float d2s = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
            if (d2s > band.hi) continue;
            if (d2s >= band.lo && !within_ff(xi, r, rc2)) continue;
            lg_pair(s, dx, dy, dz, xl, make_float4(r.v[4], r.v[5], r.v[6], r.v[7]), K);
        }
#pragma unroll
        for (int u = 0; u < kWalkChunk; ++u) qa[u] = qb[u];
    }
    float sum[3];
    s.value(sum);
    for (int a = 0; a < 3; ++a) sum[a] = group_sum<LANES>(sum[a]);
    if (live && lane == 0) atomic_max_nonneg(&smax, lg_finish(S, K, xh, xl, sum, &acc[m]));
    __syncthreads();
    if (threadIdx.x == 0 && smax) atomicMax(&ctl[kCtlAmax + (step & 1)], smax);
}

// Step `step`: x += a (h/32)/max|a| and the projection back inside the body (the
// update of Eq. 8 with dt = 0.25 sqrt(h/max|a|)), per slot; refreshes the slot's
// float32 copies and takes the largest displacement since the build.
__global__ void __launch_bounds__(256) k_relax_update_skin(int64_t n, const float4* __restrict__ acc,
                                                          const float4* __restrict__ p32,
                                                          const float4* __restrict__ lo, float4* __restrict__ rec,
                                                          Spheres S, RelaxK K,
                                                          unsigned* __restrict__ ctl, int step,
                                                          const int* __restrict__ flags) {
    __shared__ unsigned smax;
    __shared__ int skip;
    if (threadIdx.x == 0) {
        smax = 0u;
        skip = relax_halted(flags);
    }
    __syncthreads();
    if (skip) return;
    int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (m < n) {
        float am = __uint_as_float(ctl[kCtlAmax + (step & 1)]);
        const float4 ph = rec[2 * m], pl = rec[2 * m + 1];
        float xh[3] = {ph.x, ph.y, ph.z}, xl[3] = {pl.x, pl.y, pl.z}, g[3];
        if (am > 0.0f) {
            float sc = (K.h_f * 0.03125f) / am;         // a dt^2/2 = a (h/32)/max|a|
            float4 a = acc[m];
            ff_add(xh[0], xl[0], a.x * sc);
            ff_add(xh[1], xl[1], a.y * sc);
            ff_add(xh[2], xl[2], a.z * sc);
        }
        float phi = sdf32(S, xh, xl, g);
        if (phi > -0.5f * K.dp_f) {
            float sh = phi + 0.5f * K.dp_f;
            for (int c = 0; c < 3; ++c) ff_add(xh[c], xl[c], -(sh * g[c]));
        }
        float4 b = p32[m], bl = lo[m];
        rec[2 * m] = make_float4(xh[0], xh[1], xh[2], ph.w);
        rec[2 * m + 1] = make_float4(xl[0], xl[1], xl[2], pl.w);
        float ex = (xh[0] - b.x) + (xl[0] - bl.x);
        float ey = (xh[1] - b.y) + (xl[1] - bl.y);
        float ez = (xh[2] - b.z) + (xl[2] - bl.z);
        float d = sqrtf(ex * ex + ey * ey + ez * ez);
        atomicMax(&smax, isfinite(d) ? __float_as_uint(d) : 0x7f800000u);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (smax) atomicMax(&ctl[kCtlDisp + ((step + 1) & 1)], smax);
        if (blockIdx.x == 0) ctl[kCtlAmax + ((step + 1) & 1)] = 0u;
    }
}

__global__ void k_widen_acc(const float4* __restrict__ acc, int64_t n, double* __restrict__ out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float4 a = acc[i];
    out[i] = a.x;
    out[n + i] = a.y;
    out[2 * n + i] = a.z;
}

// ---------------------------------------------------------------- host helpers
int check_relax(const sph_relax_params* p) {
    if (!p) return SPH_ERR_ARG;
    int s = sph_check_domain(&p->dom);
    if (s) return s;
    if (p->dom.periodic_mask != 0) return SPH_ERR_ARG;   // a body: no periodic axes
    if (p->dom.dim != 2 && p->dom.dim != 3) return SPH_ERR_ARG;
    if (p->kernel == SPH_LAGUERRE_GAUSS) {
        if (p->dom.kappa != 2.0) return SPH_ERR_ARG;     // Eq. 8's support
    } else if (p->kernel != SPH_WENDLAND_C2) {
        return SPH_ERR_ARG;
    }
    if (p->precision != SPH_FP64 && p->precision != SPH_FP32_KAHAN) return SPH_ERR_ARG;
    // the float32 forms: 3D Laguerre-Gauss only
    if (p->precision == SPH_FP32_KAHAN && (p->dom.dim != 3 || p->kernel != SPH_LAGUERRE_GAUSS)) return SPH_ERR_ARG;
    if (p->n_spheres < 1 || p->n_spheres > SPH_MAX_SPHERES) return SPH_ERR_ARG;
    if (!(p->dp > 0.0) || !(p->rho > 0.0) || !(p->p0 > 0.0)) return SPH_ERR_ARG;
    return SPH_OK;
}

// Legendre nodes by Newton's method on P_n (three-term recurrence), mapped to [0, 1];
// weights 1 / ((1 - x^2) P_n'(x)^2) (half the [-1, 1] weights).
void gauss_legendre01(int n, double* u, double* w) {
    for (int i = 0; i < n; ++i) {
        double x = cos(SPH_PI * (i + 0.75) / (n + 0.5)), dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = x;
            for (int k = 2; k <= n; ++k) {
                double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = n * (x * p1 - p0) / (x * x - 1.0);
            double dx = p1 / dp;
            x -= dx;
            if (fabs(dx) < 1e-16) break;
        }
        // ascending order of the nodes
        u[n - 1 - i] = 0.5 * (x + 1.0);
        w[n - 1 - i] = 1.0 / ((1.0 - x * x) * dp * dp);
    }
}

int ensure_gauss_legendre(sph_ctx* ctx) {
    static std::mutex mu;
    static std::set<int> done;
    std::lock_guard<std::mutex> lock(mu);
    if (done.count(ctx->device)) return SPH_OK;
    double u[kGL], w[kGL];
    gauss_legendre01(kGL, u, w);
    SPH_CUDA(ctx, cudaMemcpyToSymbol(c_gl_u, u, sizeof(u)));
    SPH_CUDA(ctx, cudaMemcpyToSymbol(c_gl_w, w, sizeof(w)));
    done.insert(ctx->device);
    return SPH_OK;
}

Spheres make_spheres(const sph_relax_params* p) {
    Spheres S;
    S.count = p->n_spheres;
    for (int k = 0; k < SPH_MAX_SPHERES; ++k) {
        for (int c = 0; c < 3; ++c) {
            double v = k < S.count ? p->spheres[4 * k + c] : 0.0;
            S.c[k][c] = v;
            S.ch[k][c] = (float)v;
            S.cl[k][c] = (float)(v - (double)S.ch[k][c]);
        }
        S.r[k] = k < S.count ? p->spheres[4 * k + 3] : 0.0;
        S.rf[k] = (float)S.r[k];
    }
    return S;
}

RelaxK make_relax_consts(const sph_relax_params* p) {
    RelaxK K;
    const int d = p->dom.dim;
    const double h = p->dom.h;
    const double hd = d == 2 ? h * h : h * h * h;
    const double hd2 = hd * h * h;
    K.h = h;
    K.dp = p->dp;
    K.scale = 2.0 * p->p0 / p->rho;
    K.kernel = p->kernel;
    K.gcoef_lg = -lg_alpha(d) / hd2 / 3.0;
    K.gcoef_tw = -5.0 * wendland_alpha(d) / hd2;
    K.gcoef = p->kernel == SPH_WENDLAND_C2 ? K.gcoef_tw : K.gcoef_lg;
    K.w_norm = (p->kernel == SPH_WENDLAND_C2 ? wendland_alpha(d) : lg_alpha(d)) / hd;
    K.rc = p->dom.kappa * h;
    K.inv_h = 1.0 / h;
    double rtw = 1.6 * h;
    K.rc2_tw = rtw * rtw;
    K.surf_coef = 2.0 * SPH_PI * lg_alpha(3) / h;
    K.gcoef_f = (float)K.gcoef;
    K.inv_h_f = (float)K.inv_h;
    K.inv_h2_f = (float)(K.inv_h * K.inv_h);
    K.scale_f = (float)K.scale;
    K.surf_coef_f = (float)K.surf_coef;
    K.h_f = (float)h;
    K.dp_f = (float)p->dp;
    return K;
}

struct RelaxLists {
    int64_t* row_ptr;
    int32_t* col;
    int64_t cap;
};

// Neighbour lists (cut-off dom.kappa*h) of the current positions into context
// scratch; capacity overflow is flagged with the step index (first one sticks).
__global__ void k_flag_capacity(const int64_t* __restrict__ row_ptr, int64_t n, int64_t cap, int step,
                                int* __restrict__ flags) {
    if (row_ptr[n] > cap) atomicCAS(&flags[FLAG_CAPACITY], 0, step + 1);
}

int build_lists(sph_ctx* ctx, const sph_domain* dom, const double* pos, cudaStream_t s, RelaxLists& L, int step) {
    CellList cl;
    int st = sph_build_cells(ctx, dom, pos, s, &cl);
    if (st) return st;
    int64_t n = dom->n;
    int32_t* row_len = (int32_t*)sph_scratch(ctx, S_ROW_LEN, (size_t)(n + 1) * 4, &st);
    if (st) return st;
    st = sph_count_neighbors(ctx, cl, pos, n, cl.grid.rc2, row_len, s);
    if (st) return st;
    st = sph_exclusive_scan_i64(ctx, row_len, L.row_ptr, n, s);
    if (st) return st;
    k_flag_capacity<<<1, 1, 0, s>>>(L.row_ptr, n, L.cap, step, ctx->flags);
    st = sph_fill_neighbors(ctx, cl, pos, n, cl.grid.rc2, L.row_ptr, L.col, L.cap, s);
    return st;
}

int ensure_lists(sph_ctx* ctx, int64_t n, int64_t cap, RelaxLists& L) {
    int st = SPH_OK;
    L.row_ptr = (int64_t*)sph_scratch(ctx, S_RELAX_ROWPTR, (size_t)(n + 1) * 8, &st);
    L.col = (int32_t*)sph_scratch(ctx, S_RELAX_COL, (size_t)cap * 4, &st);
    L.cap = cap;
    return st;
}

// Default capacity: 128 neighbours per particle (a relaxed 3D body at h = 1.3 dp
// and cut-off 2h has about 74), regrown on overflow.
int64_t g_default_per_particle = 128;

// float32 acceleration by the cell sweep: cells of edge >= h (half the LG support),
// the neighbours of a particle within two cells of its own along each axis.
int acc_cells(sph_ctx* ctx, const sph_relax_params* p, const double* pos, const double* vol, const Spheres& S,
              const RelaxK& K, float4* acc, unsigned* amax, cudaStream_t s) {
    CellList cl;
    sph_domain half = p->dom;
    half.kappa = 0.5 * p->dom.kappa;
    int st = sph_build_cells(ctx, &half, pos, s, &cl);
    if (st) return st;
    const double rc = p->dom.kappa * p->dom.h;
    int64_t n = p->dom.n;
    float4* lo = (float4*)sph_scratch(ctx, S_MISC1, (size_t)n * 16, &st);
    if (st) return st;
    k_relax_pack_lo<<<grid_for(n, 256), 256, 0, s>>>(pos, vol, n, cl.sorted, cl.p32, lo);
    k_relax_acc_cells<2><<<grid_for(n, 256), 256, 0, s>>>(cl.p32, lo, cl.cell_start, cl.grid,
                                                          (const unsigned*)cl.band, rc * rc, pos, n, S, K, acc,
                                                          amax);
    SPH_LAUNCH_CHECK(ctx);
    return SPH_OK;
}

int read_capacity_flag(sph_ctx* ctx, cudaStream_t s, int* step_failed, int64_t* required, const RelaxLists& L,
                       int64_t n) {
    int* hf = (int*)ctx->pinned;
    int64_t* hp = (int64_t*)ctx->pinned;
    SPH_CUDA(ctx, cudaMemcpyAsync(hf, ctx->flags, FLAG_COUNT * sizeof(int), cudaMemcpyDeviceToHost, s));
    SPH_CUDA(ctx, cudaMemcpyAsync(hp + 8, L.row_ptr + n, 8, cudaMemcpyDeviceToHost, s));
    SPH_CUDA(ctx, cudaStreamSynchronize(s));
    *step_failed = hf[FLAG_CAPACITY];
    *required = hp[8];
    if (hf[FLAG_BAD_INPUT]) {
        SPH_CUDA(ctx, cudaMemsetAsync(ctx->flags, 0, FLAG_COUNT * sizeof(int), s));
        return SPH_ERR_ARG;
    }
    return SPH_OK;
}

// Default list capacity of the float32 skin list (entries per slot), regrown on
// overflow; steps issued between two reads of the status flags.
constexpr int kSkinCap = 128;
// Reach of the list build's cell sweep: cells of edge (2h + skin) / kBuildReach.
constexpr int kBuildReach = 2;
constexpr int kSkinBatch = 16;   // at most; after a rebuild, about the last list's lifetime

template <int LANES>
void walk(const float4* rec, const int32_t* col, const int32_t* rowlen, int cap, int64_t n, const unsigned* absmax,
          double lmax, double rc2, float skin, const Spheres& S, const RelaxK& K, float4* acc, unsigned* ctl, int step,
          int* flags, cudaStream_t s) {
    k_relax_walk<LANES><<<grid_for(n * LANES, 256), 256, 0, s>>>(rec, col, rowlen, cap, n, absmax, lmax, rc2, skin, S,
                                                                 K, acc, ctl, step, flags);
}

// float32 steps on the skin list.  Steps are issued in batches without host
// synchronisation; after a batch the flags say whether the list overflowed at a
// build (nothing ran: regrow and rebuild) or went stale at some step (the steps
// from there on were no-ops: rebuild at the current positions and resume there).
int relax_steps_skin(sph_ctx* ctx, const sph_relax_params* p, double* pos, const double* vol, int nsteps,
                     const Spheres& S, const RelaxK& K, cudaStream_t s) {
    const int64_t n = p->dom.n;
    const double h = p->dom.h, rc = p->dom.kappa * h, skin = ctx->relax_skin * h;
    sph_domain cells = p->dom;
    cells.kappa = (rc + skin) / (kBuildReach * h);   // cells of edge >= (2h + skin) / reach
    const int64_t slots = (n + 31) / 32 * 32;
    int st = SPH_OK;
    unsigned* ctl = (unsigned*)sph_scratch(ctx, S_RELAX_AMAX, 64, &st);
    float4* acc = (float4*)sph_scratch(ctx, S_RELAX_ACC, (size_t)n * 16, &st);
    float4* rec = (float4*)sph_scratch(ctx, S_MISC0, (size_t)n * 32, &st);
    float4* lo = (float4*)sph_scratch(ctx, S_MISC1, (size_t)n * 16, &st);
    int32_t* rowlen = (int32_t*)sph_scratch(ctx, S_RELAX_ROWPTR, (size_t)n * 4, &st);
    if (st) return st;
    int64_t have = (int64_t)(ctx->slot_bytes[S_RELAX_COL] / ((size_t)slots * 4));
    int cap = (int)std::min<int64_t>(std::max<int64_t>(have, kSkinCap), 1 << 16);
    const float skin_f = (float)(skin * (1.0 - 1e-3));
    int* hf = (int*)ctx->pinned;
    SPH_CUDA(ctx, cudaMemsetAsync(ctx->flags, 0, FLAG_COUNT * sizeof(int), s));
    CellList cl;
    int32_t* col = nullptr;
    bool build = true, moved = false;     // moved: rec holds steps not yet in pos
    int done = 0, regrow = 0, built_at = 0, batch = kSkinBatch;
    while (done < nsteps) {
        if (build) {
            col = (int32_t*)sph_scratch(ctx, S_RELAX_COL, (size_t)slots * cap * 4, &st);
            if (st) return st;
            int t = sph_timer_begin(ctx, SPH_TIMER_NEIGHBORS, s);
            if (moved) k_relax_scatter_pos<<<grid_for(n, 256), 256, 0, s>>>(rec, cl.sorted, n, pos);
            moved = false;
            st = sph_build_cells(ctx, &cells, pos, s, &cl);
            if (st) return st;
            k_relax_pack_lo<<<grid_for(n, 256), 256, 0, s>>>(pos, vol, n, cl.sorted, cl.p32, lo);
            SPH_CUDA(ctx, cudaMemsetAsync(ctl, 0, 64, s));
            k_relax_skin_build<kBuildReach><<<grid_for(n, 256), 256, 0, s>>>(cl.p32, lo, cl.cell_start, cl.grid,
                                                                   (const unsigned*)cl.band, (rc + skin) * (rc + skin),
                                                                   pos, n, cap, col, rowlen, rec, ctl, done,
                                                                   ctx->flags);
            sph_timer_end(ctx, t, s);
            SPH_LAUNCH_CHECK(ctx);
            built_at = done;
        }
        const int end = std::min(nsteps, done + batch);
        const unsigned* absmax = (const unsigned*)cl.band;
        for (int k = done; k < end; ++k) {
            int t = sph_timer_begin(ctx, SPH_TIMER_RELAX_ACCEL, s);
            switch (ctx->lanes[SPH_PASS_RELAX]) {
                case 1: walk<1>(rec, col, rowlen, cap, n, absmax, skin, rc * rc, skin_f, S, K, acc, ctl, k, ctx->flags, s); break;
                case 2: walk<2>(rec, col, rowlen, cap, n, absmax, skin, rc * rc, skin_f, S, K, acc, ctl, k, ctx->flags, s); break;
                case 8: walk<8>(rec, col, rowlen, cap, n, absmax, skin, rc * rc, skin_f, S, K, acc, ctl, k, ctx->flags, s); break;
                default: walk<4>(rec, col, rowlen, cap, n, absmax, skin, rc * rc, skin_f, S, K, acc, ctl, k, ctx->flags, s); break;
            }
            sph_timer_end(ctx, t, s);
            t = sph_timer_begin(ctx, SPH_TIMER_RELAX_UPDATE, s);
            k_relax_update_skin<<<grid_for(n, 256), 256, 0, s>>>(n, acc, cl.p32, lo, rec, S, K,
                                                                 ctl, k, ctx->flags);
            sph_timer_end(ctx, t, s);
            SPH_LAUNCH_CHECK(ctx);
        }
        moved = moved || end > done;
        SPH_CUDA(ctx, cudaMemcpyAsync(hf, ctx->flags, FLAG_COUNT * sizeof(int), cudaMemcpyDeviceToHost, s));
        SPH_CUDA(ctx, cudaMemcpyAsync(hf + 16, ctl + kCtlNeed, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
        SPH_CUDA(ctx, cudaStreamSynchronize(s));
        const int bad = hf[FLAG_BAD_INPUT], over = hf[FLAG_CAPACITY], stale = hf[FLAG_STALE];
        const int need = hf[16];
        if (bad || over || stale) SPH_CUDA(ctx, cudaMemsetAsync(ctx->flags, 0, FLAG_COUNT * sizeof(int), s));
        if (bad) return SPH_ERR_ARG;     // non-finite positions (pos holds them)
        if (over) {                       // the build overflowed: no step ran
            if (++regrow > 4 || need >= (1 << 16)) return SPH_ERR_CAPACITY;
            cap = (need + need / 8 + 8 + 7) / 8 * 8;
            build = true;
            continue;
        }
        if (stale) {                      // steps stale - 1 .. end - 1 were no-ops
            done = stale - 1;
            const int life = done - built_at;
            batch = std::max(2, std::min(kSkinBatch, life + life / 4 + 1));
            build = true;
            continue;
        }
        done = end;
        build = false;
    }
    if (moved) k_relax_scatter_pos<<<grid_for(n, 256), 256, 0, s>>>(rec, cl.sorted, n, pos);
    SPH_LAUNCH_CHECK(ctx);
    return SPH_OK;
}

}  // namespace

extern "C" int sph_relax_step(sph_ctx* ctx, const sph_relax_params* p, double* pos, const double* vol, int nsteps,
                              void* stream) {
    if (!ctx || nsteps < 0) return SPH_ERR_ARG;
    int st = check_relax(p);
    if (st) return st;
    int64_t n = p->dom.n;
    if (n == 0 || nsteps == 0) return SPH_OK;
    if (!pos || !vol) return SPH_ERR_ARG;
    cudaStream_t s = as_stream(stream);
    Spheres S = make_spheres(p);
    RelaxK K = make_relax_consts(p);
    st = ensure_gauss_legendre(ctx);
    if (st) return st;
    if (p->precision == SPH_FP32_KAHAN && ctx->relax_skin > 0.0)
        return relax_steps_skin(ctx, p, pos, vol, nsteps, S, K, s);
    if (p->precision == SPH_FP32_KAHAN) {
        unsigned* amax = (unsigned*)sph_scratch(ctx, S_RELAX_AMAX, 64, &st);
        float4* acc = (float4*)sph_scratch(ctx, S_RELAX_ACC, (size_t)n * 16, &st);
        if (st) return st;
        SPH_CUDA(ctx, cudaMemsetAsync(ctx->flags, 0, FLAG_COUNT * sizeof(int), s));
        for (int k = 0; k < nsteps; ++k) {
            SPH_CUDA(ctx, cudaMemsetAsync(amax, 0, 64, s));
            int t = sph_timer_begin(ctx, SPH_TIMER_RELAX_ACCEL, s);
            st = acc_cells(ctx, p, pos, vol, S, K, acc, amax, s);
            if (st) return st;
            sph_timer_end(ctx, t, s);
            t = sph_timer_begin(ctx, SPH_TIMER_RELAX_UPDATE, s);
            k_relax_update32<<<grid_for(n, 256), 256, 0, s>>>(pos, n, acc, amax, S, K, ctx->flags);
            sph_timer_end(ctx, t, s);
            SPH_LAUNCH_CHECK(ctx);
        }
        int* hf = (int*)ctx->pinned;
        SPH_CUDA(ctx, cudaMemcpyAsync(hf, ctx->flags, FLAG_COUNT * sizeof(int), cudaMemcpyDeviceToHost, s));
        SPH_CUDA(ctx, cudaStreamSynchronize(s));
        if (hf[FLAG_BAD_INPUT]) {
            SPH_CUDA(ctx, cudaMemsetAsync(ctx->flags, 0, FLAG_COUNT * sizeof(int), s));
            return SPH_ERR_ARG;
        }
        return SPH_OK;
    }
    int64_t cap = ctx->slot_bytes[S_RELAX_COL] / 4;
    if (cap < n * g_default_per_particle) cap = n * g_default_per_particle;
    RelaxLists L;
    st = ensure_lists(ctx, n, cap, L);
    if (st) return st;
    unsigned* amax = (unsigned*)sph_scratch(ctx, S_RELAX_AMAX, 64, &st);
    if (st) return st;
    unsigned long long* amax_d = (unsigned long long*)(amax + 4);
    double* acc = (double*)sph_scratch(ctx, S_RELAX_ACC, (size_t)n * 24, &st);
    if (st) return st;
    SPH_CUDA(ctx, cudaMemsetAsync(ctx->flags, 0, FLAG_COUNT * sizeof(int), s));
    int done = 0;
    for (int attempt = 0; attempt < 8 && done < nsteps; ++attempt) {
        for (int k = done; k < nsteps; ++k) {
            int t = sph_timer_begin(ctx, SPH_TIMER_NEIGHBORS, s);
            st = build_lists(ctx, &p->dom, pos, s, L, k);
            if (st) return st;
            sph_timer_end(ctx, t, s);
            SPH_CUDA(ctx, cudaMemsetAsync(amax, 0, 64, s));
            t = sph_timer_begin(ctx, SPH_TIMER_RELAX_ACCEL, s);
            if (p->dom.dim == 2) {
                k_relax_acc64<2><<<grid_for(n, 128), 128, 0, s>>>(pos, vol, n, L.row_ptr, L.col, S, K, acc, amax,
                                                                  ctx->flags);
                k_amax64_exact<2><<<grid_for(n, 256), 256, 0, s>>>(acc, n, amax, amax_d, ctx->flags);
            } else {
                k_relax_acc64<3><<<grid_for(n, 128), 128, 0, s>>>(pos, vol, n, L.row_ptr, L.col, S, K, acc, amax,
                                                                  ctx->flags);
                k_amax64_exact<3><<<grid_for(n, 256), 256, 0, s>>>(acc, n, amax, amax_d, ctx->flags);
            }
            sph_timer_end(ctx, t, s);
            t = sph_timer_begin(ctx, SPH_TIMER_RELAX_UPDATE, s);
            if (p->dom.dim == 2)
                k_relax_update64<2><<<grid_for(n, 256), 256, 0, s>>>(pos, n, acc, amax_d, S, K, ctx->flags);
            else
                k_relax_update64<3><<<grid_for(n, 256), 256, 0, s>>>(pos, n, acc, amax_d, S, K, ctx->flags);
            sph_timer_end(ctx, t, s);
            SPH_LAUNCH_CHECK(ctx);
        }
        int failed = 0;
        int64_t required = 0;
        st = read_capacity_flag(ctx, s, &failed, &required, L, n);
        if (st) return st;
        if (!failed) { done = nsteps; break; }
        done = failed - 1;
        SPH_CUDA(ctx, cudaMemsetAsync(ctx->flags, 0, FLAG_COUNT * sizeof(int), s));
        st = ensure_lists(ctx, n, required + required / 4 + 1024, L);
        if (st) return st;
    }
    return done == nsteps ? SPH_OK : SPH_ERR_CAPACITY;
}

extern "C" int sph_relax_accel(sph_ctx* ctx, const sph_relax_params* p, const double* pos, const double* vol,
                               double* acc_out, void* stream) {
    if (!ctx) return SPH_ERR_ARG;
    int st = check_relax(p);
    if (st) return st;
    int64_t n = p->dom.n;
    if (n == 0) return SPH_OK;
    if (!pos || !vol || !acc_out) return SPH_ERR_ARG;
    cudaStream_t s = as_stream(stream);
    Spheres S = make_spheres(p);
    RelaxK K = make_relax_consts(p);
    st = ensure_gauss_legendre(ctx);
    if (st) return st;
    if (p->precision == SPH_FP32_KAHAN) {
        unsigned* amax = (unsigned*)sph_scratch(ctx, S_RELAX_AMAX, 64, &st);
        float4* acc = (float4*)sph_scratch(ctx, S_RELAX_ACC, (size_t)n * 16, &st);
        if (st) return st;
        SPH_CUDA(ctx, cudaMemsetAsync(amax, 0, 64, s));
        st = acc_cells(ctx, p, pos, vol, S, K, acc, amax, s);
        if (st) return st;
        k_widen_acc<<<grid_for(n, 256), 256, 0, s>>>(acc, n, acc_out);
        SPH_LAUNCH_CHECK(ctx);
        int* hf = (int*)ctx->pinned;
        SPH_CUDA(ctx, cudaMemcpyAsync(hf, ctx->flags, FLAG_COUNT * sizeof(int), cudaMemcpyDeviceToHost, s));
        SPH_CUDA(ctx, cudaMemsetAsync(ctx->flags, 0, FLAG_COUNT * sizeof(int), s));
        SPH_CUDA(ctx, cudaStreamSynchronize(s));
        return hf[FLAG_BAD_INPUT] ? SPH_ERR_ARG : SPH_OK;
    }
    int64_t cap = n * g_default_per_particle;
    RelaxLists L;
    for (int attempt = 0; attempt < 4; ++attempt) {
        st = ensure_lists(ctx, n, cap, L);
        if (st) return st;
        SPH_CUDA(ctx, cudaMemsetAsync(ctx->flags, 0, FLAG_COUNT * sizeof(int), s));
        st = build_lists(ctx, &p->dom, pos, s, L, 0);
        if (st) return st;
        int failed = 0;
        int64_t required = 0;
        st = read_capacity_flag(ctx, s, &failed, &required, L, n);
        if (st) return st;
        if (!failed) break;
        cap = required + required / 4 + 1024;
        SPH_CUDA(ctx, cudaMemsetAsync(ctx->flags, 0, FLAG_COUNT * sizeof(int), s));
    }
    unsigned* amax = (unsigned*)sph_scratch(ctx, S_RELAX_AMAX, 64, &st);
    if (st) return st;
    SPH_CUDA(ctx, cudaMemsetAsync(amax, 0, 64, s));
    if (p->dom.dim == 2)
        k_relax_acc64<2><<<grid_for(n, 128), 128, 0, s>>>(pos, vol, n, L.row_ptr, L.col, S, K, acc_out, amax,
                                                          ctx->flags);
    else
        k_relax_acc64<3><<<grid_for(n, 128), 128, 0, s>>>(pos, vol, n, L.row_ptr, L.col, S, K, acc_out, amax,
                                                          ctx->flags);
    SPH_LAUNCH_CHECK(ctx);
    return SPH_OK;
}

// The Laguerre-Gauss residual from the float32 pair sums: for a particle with
// phi < -2h the surface term of Eq. 7 vanishes (its support lies inside the body), so
// sum_j grad W_ij V_j = -a_i / scale with a_i the float32 acceleration of one cell sweep
// (compensated sums); h^2 |.|^2 and the count are reduced in float64 in a fixed order.
__global__ void k_residual_from_acc(const float4* __restrict__ acc, const double* __restrict__ pos, int64_t n,
                                    Spheres S, RelaxK K, double* __restrict__ partial) {
    __shared__ double sh[2][256];
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double e = 0.0, cnt = 0.0;
    if (i < n) {
        double xi[3] = {pos[i], pos[n + i], pos[2 * n + i]}, g[3];
        if (sdf64<3>(S, xi, g) < -2.0 * K.h) {
            const float4 a = acc[i];
            const double sx = (double)a.x / K.scale, sy = (double)a.y / K.scale, sz = (double)a.z / K.scale;
            e = K.h * K.h * (sx * sx + sy * sy + sz * sz);
            cnt = 1.0;
        }
    }
    sh[0][threadIdx.x] = e;
    sh[1][threadIdx.x] = cnt;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) {
            sh[0][threadIdx.x] += sh[0][threadIdx.x + o];
            sh[1][threadIdx.x] += sh[1][threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        partial[3 * blockIdx.x] = sh[0][0];
        partial[3 * blockIdx.x + 1] = 0.0;
        partial[3 * blockIdx.x + 2] = sh[1][0];
    }
}

extern "C" int sph_relax_residual_fp32(sph_ctx* ctx, const sph_relax_params* p, const double* pos, const double* vol,
                                       double* out_host, void* stream) {
    if (!ctx || !out_host) return SPH_ERR_ARG;
    int st = check_relax(p);
    if (st) return st;
    if (p->dom.dim != 3 || p->kernel != SPH_LAGUERRE_GAUSS) return SPH_ERR_ARG;
    const int64_t n = p->dom.n;
    out_host[0] = out_host[2] = 0.0;
    out_host[1] = NAN;
    if (n == 0) return SPH_OK;
    if (!pos || !vol) return SPH_ERR_ARG;
    cudaStream_t s = as_stream(stream);
    Spheres S = make_spheres(p);
    RelaxK K = make_relax_consts(p);
    st = ensure_gauss_legendre(ctx);
    if (st) return st;
    unsigned* amax = (unsigned*)sph_scratch(ctx, S_RELAX_AMAX, 64, &st);
    float4* acc = (float4*)sph_scratch(ctx, S_RELAX_ACC, (size_t)n * 16, &st);
    if (st) return st;
    SPH_CUDA(ctx, cudaMemsetAsync(amax, 0, 64, s));
    st = acc_cells(ctx, p, pos, vol, S, K, acc, amax, s);
    if (st) return st;
    const int nb = (int)grid_for(n, 256);
    double* partial = (double*)sph_scratch(ctx, S_RED_PARTIAL, (size_t)nb * 3 * 8 + 64, &st);
    if (st) return st;
    double* out_d = partial + (size_t)nb * 3;
    k_residual_from_acc<<<nb, 256, 0, s>>>(acc, pos, n, S, K, partial);
    k_sum_partials<<<1, 256, 0, s>>>(partial, nb, out_d);
    SPH_LAUNCH_CHECK(ctx);
    double* hp = (double*)ctx->pinned;
    SPH_CUDA(ctx, cudaMemcpyAsync(hp + 32, out_d, 3 * sizeof(double), cudaMemcpyDeviceToHost, s));
    int* hf = (int*)ctx->pinned;
    SPH_CUDA(ctx, cudaMemcpyAsync(hf, ctx->flags, FLAG_COUNT * sizeof(int), cudaMemcpyDeviceToHost, s));
    SPH_CUDA(ctx, cudaMemsetAsync(ctx->flags, 0, FLAG_COUNT * sizeof(int), s));
    SPH_CUDA(ctx, cudaStreamSynchronize(s));
    if (hf[FLAG_BAD_INPUT]) return SPH_ERR_ARG;
    const double m = hp[34];
    if (!isfinite(hp[32])) return SPH_ERR_NONFINITE;
    out_host[2] = m;
    if (m > 0.0) out_host[0] = sqrt(hp[32] / m);
    return SPH_OK;
}

extern "C" int sph_relax_residual(sph_ctx* ctx, const sph_relax_params* p, const double* pos, const double* vol,
                                  double* out_host, void* stream) {
    if (!ctx || !out_host) return SPH_ERR_ARG;
    int st = check_relax(p);
    if (st) return st;
    int64_t n = p->dom.n;
    out_host[0] = out_host[1] = out_host[2] = 0.0;
    if (n == 0) return SPH_OK;
    if (!pos || !vol) return SPH_ERR_ARG;
    cudaStream_t s = as_stream(stream);
    Spheres S = make_spheres(p);
    RelaxK K = make_relax_consts(p);
    sph_domain dom = p->dom;
    dom.kappa = 2.0;
    int64_t cap = n * g_default_per_particle;
    RelaxLists L;
    for (int attempt = 0; attempt < 4; ++attempt) {
        st = ensure_lists(ctx, n, cap, L);
        if (st) return st;
        SPH_CUDA(ctx, cudaMemsetAsync(ctx->flags, 0, FLAG_COUNT * sizeof(int), s));
        st = build_lists(ctx, &dom, pos, s, L, 0);
        if (st) return st;
        int failed = 0;
        int64_t required = 0;
        st = read_capacity_flag(ctx, s, &failed, &required, L, n);
        if (st) return st;
        if (!failed) break;
        cap = required + required / 4 + 1024;
        SPH_CUDA(ctx, cudaMemsetAsync(ctx->flags, 0, FLAG_COUNT * sizeof(int), s));
    }
    int nb = (int)grid_for(n, 256);
    double* partial = (double*)sph_scratch(ctx, S_RED_PARTIAL, (size_t)nb * 3 * 8 + 64, &st);
    if (st) return st;
    double* out_d = partial + (size_t)nb * 3;
    if (p->dom.dim == 2) k_relax_residual<2><<<nb, 256, 0, s>>>(pos, vol, n, L.row_ptr, L.col, S, K, partial);
    else k_relax_residual<3><<<nb, 256, 0, s>>>(pos, vol, n, L.row_ptr, L.col, S, K, partial);
    k_sum_partials<<<1, 256, 0, s>>>(partial, nb, out_d);
    SPH_LAUNCH_CHECK(ctx);
    double* hp = (double*)ctx->pinned;
    SPH_CUDA(ctx, cudaMemcpyAsync(hp + 32, out_d, 3 * sizeof(double), cudaMemcpyDeviceToHost, s));
    SPH_CUDA(ctx, cudaStreamSynchronize(s));
    double m = hp[34];
    if (!isfinite(hp[32]) || !isfinite(hp[33])) return SPH_ERR_NONFINITE;
    out_host[2] = m;
    if (m > 0.0) {
        out_host[0] = sqrt(hp[32] / m);
        out_host[1] = sqrt(hp[33] / m);
    }
    return SPH_OK;
}
