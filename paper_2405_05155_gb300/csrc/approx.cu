// x1: SPH approximations of a field and of its gradient for the error analysis
// (Sec. 2.3.3): the kernel summation sum_j f_j W_ij V_j (over the listed pairs and
// i itself; f = 1 is the normalisation condition of Eq. 3) and the weak form of
// Eq. 4 written with grad W_ij = grad_i W, sum_j (f_i + f_j) B_i grad W_ij V_j, with
// the correction matrix of Eq. 9 or with B_i = I.  Float64, one thread per particle.
#include "common.cuh"

namespace {

struct Box64 {
    double len[3], half[3];
    uint32_t periodic;
};

// Kernel value divided by alpha_d h^-d (Eqs. 6 and 8), uncut: the pairs are the
// lists' (d^2 <= (kappa h)^2).
__device__ __forceinline__ double shape(int kernel, double q) {
    if (kernel == SPH_WENDLAND_C2) {
        double t = 1.0 - 0.5 * q;
        return t * t * t * t * (2.0 * q + 1.0);
    }
    double q2 = q * q;
    return (1.0 - 0.5 * q2 + q2 * q2 / 6.0) * exp(-q2);
}

template <int DIM>
__global__ void k_field_approx(const double* __restrict__ pos, const double* __restrict__ vol,
                               const double* __restrict__ f, const int64_t* __restrict__ row_ptr,
                               const int32_t* __restrict__ col, int64_t n, Box64 box, int kernel, double inv_h,
                               double wnorm, double coef, const double* __restrict__ B, double* __restrict__ sum,
                               double* __restrict__ grad) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    constexpr int NS = DIM == 2 ? 3 : 6;
    double xi[DIM];
#pragma unroll
    for (int k = 0; k < DIM; ++k) xi[k] = pos[k * n + i];
    const double fi = f[i];
    double s = 0.0, g[DIM];
#pragma unroll
    for (int a = 0; a < DIM; ++a) g[a] = 0.0;
    for (int64_t p = row_ptr[i], e = row_ptr[i + 1]; p < e; ++p) {
        const int j = col[p];
        double r[DIM], d2 = 0.0;
#pragma unroll
        for (int k = 0; k < DIM; ++k) {
            double dx = xi[k] - pos[k * n + j];
            if ((box.periodic >> k) & 1u) {
                if (dx > box.half[k]) dx -= box.len[k];
                else if (dx < -box.half[k]) dx += box.len[k];
            }
            r[k] = dx;
            d2 += dx * dx;
        }
        const double q = sqrt(d2) * inv_h;
        const double fj = f[j], vj = vol[j];
        s += fj * (wnorm * shape(kernel, q)) * vj;
        const double gs = kernel == SPH_WENDLAND_C2 ? wendland_gs<double>(q, coef) : lg_gs<double>(q, coef);
        const double c = (fi + fj) * vj * gs;
#pragma unroll
        for (int a = 0; a < DIM; ++a) g[a] += c * r[a];
    }
    if (sum) sum[i] = s + fi * vol[i] * (wnorm * shape(kernel, 0.0));
    if (!grad) return;
    if (B) {
        double Bs[NS];
#pragma unroll
        for (int t = 0; t < NS; ++t) Bs[t] = B[t * n + i];
        double y[DIM];
        if (DIM == 2) {
            y[0] = Bs[0] * g[0] + Bs[1] * g[1];
            y[1] = Bs[1] * g[0] + Bs[2] * g[1];
        } else {
            y[0] = Bs[0] * g[0] + Bs[1] * g[1] + Bs[2] * g[DIM - 1];
            y[1] = Bs[1] * g[0] + Bs[3] * g[1] + Bs[4] * g[DIM - 1];
            y[DIM - 1] = Bs[2] * g[0] + Bs[4] * g[1] + Bs[5] * g[DIM - 1];
        }
#pragma unroll
        for (int a = 0; a < DIM; ++a) g[a] = y[a];
    }
#pragma unroll
    for (int a = 0; a < DIM; ++a) grad[a * n + i] = g[a];
}

}  // namespace

extern "C" int sph_field_approx(sph_ctx* ctx, const sph_domain* dom, int kernel, const double* pos,
                                const double* vol, const int64_t* row_ptr, const int32_t* col, const double* B,
                                const double* f, double* sum, double* grad, void* stream) {
    if (!ctx) return SPH_ERR_ARG;
    int st = sph_check_domain(dom);
    if (st) return st;
    if (kernel != SPH_WENDLAND_C2 && kernel != SPH_LAGUERRE_GAUSS) return SPH_ERR_ARG;
    const int64_t n = dom->n;
    if (n == 0 || (!sum && !grad)) return SPH_OK;
    if (!pos || !vol || !row_ptr || !col || !f) return SPH_ERR_ARG;
    cudaStream_t s = as_stream(stream);
    Box64 box;
    for (int k = 0; k < 3; ++k) { box.len[k] = dom->len[k]; box.half[k] = 0.5 * dom->len[k]; }
    box.periodic = dom->periodic_mask;
    const int d = dom->dim;
    const double h = dom->h;
    const double hd = d == 2 ? h * h : h * h * h, hd2 = hd * h * h;
    const double alpha = kernel == SPH_WENDLAND_C2 ? wendland_alpha(d) : lg_alpha(d);
    const double coef = kernel == SPH_WENDLAND_C2 ? -5.0 * alpha / hd2 : -alpha / hd2 / 3.0;
    if (d == 2)
        k_field_approx<2><<<grid_for(n, 128), 128, 0, s>>>(pos, vol, f, row_ptr, col, n, box, kernel, 1.0 / h,
                                                           alpha / hd, coef, B, sum, grad);
    else
        k_field_approx<3><<<grid_for(n, 128), 128, 0, s>>>(pos, vol, f, row_ptr, col, n, box, kernel, 1.0 / h,
                                                           alpha / hd, coef, B, sum, grad);
    SPH_LAUNCH_CHECK(ctx);
    return SPH_OK;
}
