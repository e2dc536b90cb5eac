// a4: kernel-gradient-correction matrices B_i = -(sum_j V_j r_ij (x) grad W_ij)^-1
// (Eq. 9, Sec. 2.3.2), float64, one thread per particle.
#include "common.cuh"

namespace {

struct Geo64 {
    double len[3], half[3];
    uint32_t periodic;
};

template <int DIM>
__global__ void k_kgc(const double* __restrict__ pos, const double* __restrict__ vol,
                      const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col, int64_t n,
                      Geo64 geo, int kernel, double inv_h, double coef, double* __restrict__ B,
                      uint8_t* __restrict__ fallback, unsigned long long* __restrict__ nfb) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    constexpr int NS = DIM == 2 ? 3 : 6;
    double xi[DIM];
#pragma unroll
    for (int k = 0; k < DIM; ++k) xi[k] = pos[k * n + i];
    double A[NS];
#pragma unroll
    for (int s = 0; s < NS; ++s) A[s] = 0.0;
    int64_t b = row_ptr[i], e = row_ptr[i + 1];
    for (int64_t p = b; p < e; ++p) {
        int j = col[p];
        double r[DIM];
        double d2 = 0.0;
#pragma unroll
        for (int k = 0; k < DIM; ++k) {
            double dx = xi[k] - pos[k * n + j];
            if ((geo.periodic >> k) & 1u) {
                if (dx > geo.half[k]) dx -= geo.len[k];
                else if (dx < -geo.half[k]) dx += geo.len[k];
            }
            r[k] = dx;
            d2 += dx * dx;
        }
        double q = sqrt(d2) * inv_h;
        double gs = kernel == SPH_WENDLAND_C2 ? wendland_gs<double>(q, coef) : lg_gs<double>(q, coef);
        double w = vol[j];
        int s = 0;
#pragma unroll
        for (int a = 0; a < DIM; ++a)
#pragma unroll
            for (int c = a; c < DIM; ++c) A[s++] -= w * r[a] * (gs * r[c]);
    }
    double Bv[NS];
    double det, tr;
    bool finite = true;
#pragma unroll
    for (int s = 0; s < NS; ++s) finite = finite && isfinite(A[s]);
    if (DIM == 2) {
        det = A[0] * A[2] - A[1] * A[1];
        tr = A[0] + A[2];
        Bv[0] = A[2] / det;
        Bv[1] = -A[1] / det;
        Bv[2] = A[0] / det;
    } else {
        double a00 = A[0], a01 = A[1], a02 = A[2], a11 = A[3], a12 = A[4], a22 = A[5];
        double c00 = a11 * a22 - a12 * a12;
        double c01 = a02 * a12 - a01 * a22;
        double c02 = a01 * a12 - a02 * a11;
        double c11 = a00 * a22 - a02 * a02;
        double c12 = a01 * a02 - a00 * a12;
        double c22 = a00 * a11 - a01 * a01;
        det = a00 * c00 + a01 * c01 + a02 * c02;
        tr = a00 + a11 + a22;
        Bv[0] = c00 / det; Bv[1] = c01 / det; Bv[2] = c02 / det;
        Bv[3] = c11 / det; Bv[4] = c12 / det; Bv[5] = c22 / det;
    }
    double m = tr / DIM;
    double bound = DIM == 2 ? 1e-8 * m * m : 1e-8 * m * m * m;
    bool ok = finite && tr > 0.0 && det > bound;
    if (!ok) {
        if (DIM == 2) { Bv[0] = 1.0; Bv[1] = 0.0; Bv[2] = 1.0; }
        else { Bv[0] = 1.0; Bv[1] = 0.0; Bv[2] = 0.0; Bv[3] = 1.0; Bv[4] = 0.0; Bv[5] = 1.0; }
        atomicAdd(nfb, 1ULL);
    }
#pragma unroll
    for (int s = 0; s < NS; ++s) B[s * n + i] = Bv[s];
    if (fallback) fallback[i] = ok ? 0 : 1;
}

}  // namespace

extern "C" int sph_kgc(sph_ctx* ctx, const sph_domain* dom, int kernel, const double* pos, const double* vol,
                       const int64_t* row_ptr, const int32_t* col, double* B, uint8_t* fallback,
                       int64_t* n_fallback_host, void* stream) {
    if (!ctx) return SPH_ERR_ARG;
    int st = sph_check_domain(dom);
    if (st) return st;
    if (kernel != SPH_WENDLAND_C2 && kernel != SPH_LAGUERRE_GAUSS) return SPH_ERR_ARG;
    int64_t n = dom->n;
    if (n > 0 && (!pos || !vol || !row_ptr || !col || !B)) return SPH_ERR_ARG;
    cudaStream_t s = as_stream(stream);
    unsigned long long* cnt = (unsigned long long*)sph_scratch(ctx, S_KGC_COUNT, 64, &st);
    if (st) return st;
    SPH_CUDA(ctx, cudaMemsetAsync(cnt, 0, 8, s));
    Geo64 geo;
    for (int k = 0; k < 3; ++k) { geo.len[k] = dom->len[k]; geo.half[k] = 0.5 * dom->len[k]; }
    geo.periodic = dom->periodic_mask;
    int d = dom->dim;
    double h = dom->h;
    double hd2 = d == 2 ? h * h * h * h : h * h * h * h * h;   // h^(d+2)
    double coef = kernel == SPH_WENDLAND_C2 ? -5.0 * wendland_alpha(d) / hd2 : -lg_alpha(d) / hd2 / 3.0;
    if (n > 0) {
        if (d == 2)
            k_kgc<2><<<grid_for(n, 128), 128, 0, s>>>(pos, vol, row_ptr, col, n, geo, kernel, 1.0 / h, coef, B,
                                                      fallback, cnt);
        else
            k_kgc<3><<<grid_for(n, 128), 128, 0, s>>>(pos, vol, row_ptr, col, n, geo, kernel, 1.0 / h, coef, B,
                                                      fallback, cnt);
        SPH_LAUNCH_CHECK(ctx);
    }
    if (n_fallback_host) {
        int64_t* hp = (int64_t*)ctx->pinned;
        SPH_CUDA(ctx, cudaMemcpyAsync(hp + 16, cnt, 8, cudaMemcpyDeviceToHost, s));
        SPH_CUDA(ctx, cudaStreamSynchronize(s));
        *n_fallback_host = hp[16];
    }
    return SPH_OK;
}
