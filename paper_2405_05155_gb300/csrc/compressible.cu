// x2: Riemann-based Eulerian SPH for compressible flow (Sec. 3.1): the mass, momentum
// and energy rows of Eq. 18 with the ideal-gas EOS (Eqs. 15-16) and the HLLC solver with
// the dissipation limiter (Eqs. 20-24), float64, one thread per particle over its CSR
// row, forward Euler in time.  Readings (see include/sph.h): the star density and
// energy use the normal velocity u where |v| is printed; the limited p* adds the two
// impedance terms; the interface state follows the wave fan, the star state when S_l
// and S_r cross, the star mean at u* = 0.
#include "common.cuh"

namespace {

struct CompK {
    double gamma, eta, coef, inv_h, dt;
    double len[3], half[3];
    uint32_t periodic;
};

template <int DIM>
struct Prim {
    double rho, v[DIM], p, c, E;
};

template <int DIM>
__device__ __forceinline__ Prim<DIM> prim(const double* rho, const double* mom, const double* E, int64_t n,
                                          int64_t i, double gamma) {
    Prim<DIM> s;
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

// Interface state (rho_s, v_s, E_s, p_s) of the limited HLLC solver along nrm (i -> j).
template <int DIM>
__device__ __forceinline__ void hllc(const Prim<DIM>& L, const Prim<DIM>& R, const double* nrm, double eta,
                                     double& rho_s, double* v_s, double& E_s, double& p_s) {
    double ul = 0.0, ur = 0.0;
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
        ul += L.v[a] * nrm[a];
        ur += R.v[a] * nrm[a];
    }
    const double sl = ul - L.c, sr = ur + R.c;
    const double cbar = 0.5 * (L.c + R.c);
    const double beta = fmin(eta * fmax((ul - ur) / cbar, 0.0), 1.0);
    const double zl = L.rho * L.c, zr = R.rho * R.c;
    const double ustar = (zl * ul + zr * ur + beta * beta * (L.p - R.p)) / (zl + zr);
    const double pstar = 0.5 * (L.p + R.p) + 0.5 * beta * (zr * (ustar - ur) + zl * (ul - ustar));
    const bool left = sl >= 0.0 && sr > 0.0;
    const bool right = sr <= 0.0 && sl < 0.0;
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
    const double rho_sl = L.rho * (sl - ul) / (sl - ustar);
    const double rho_sr = R.rho * (sr - ur) / (sr - ustar);
    const double E_sl = ((sl - ul) * L.E - L.p * ul + pstar * ustar) / (sl - ustar);
    const double E_sr = ((sr - ur) * R.E - R.p * ur + pstar * ustar) / (sr - ustar);
    if (ustar > 0.0) { rho_s = rho_sl; E_s = E_sl; }
    else if (ustar < 0.0) { rho_s = rho_sr; E_s = E_sr; }
    else { rho_s = 0.5 * (rho_sl + rho_sr); E_s = 0.5 * (E_sl + E_sr); }
    p_s = pstar;
#pragma unroll
    for (int a = 0; a < DIM; ++a) v_s[a] = ustar * nrm[a] + 0.5 * (L.v[a] + R.v[a]) - 0.5 * (ul + ur) * nrm[a];
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
    const Prim<DIM> Pi = prim<DIM>(rho, mom, E, n, i, K.gamma);
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
        const Prim<DIM> Pj = prim<DIM>(rho, mom, E, n, j, K.gamma);
        double rho_s, v_s[DIM], E_s, p_s;
        hllc<DIM>(Pi, Pj, nrm, K.eta, rho_s, v_s, E_s, p_s);
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

int check(const sph_compressible_params* p, const sph_compressible_state* st) {
    if (!p || !st) return SPH_ERR_ARG;
    int r = sph_check_domain(&p->dom);
    if (r) return r;
    if (p->precision != SPH_FP64) return SPH_ERR_ARG;
    if (!(p->gamma > 1.0) || !(p->eta >= 0.0) || !(p->dt >= 0.0)) return SPH_ERR_ARG;
    if (p->dom.n > 0 && (!st->row_ptr || !st->col || !st->pos || !st->vol || !st->B || !st->rho || !st->mom ||
                         !st->E))
        return SPH_ERR_ARG;
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

}  // namespace

extern "C" int sph_compressible_rates(sph_ctx* ctx, const sph_compressible_params* p,
                                      const sph_compressible_state* st, double* drho, double* dmom, double* dE,
                                      void* stream) {
    if (!ctx) return SPH_ERR_ARG;
    int r = check(p, st);
    if (r) return r;
    if (p->dom.n == 0) return SPH_OK;
    if (!drho || !dmom || !dE) return SPH_ERR_ARG;
    launch_rates(p, st, consts(p), drho, dmom, dE, as_stream(stream));
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
    const int dim = p->dom.dim;
    double* rates = (double*)sph_scratch(ctx, S_MISC2, (size_t)n * (dim + 2) * 8, &r);
    if (r) return r;
    double *drho = rates, *dmom = rates + n, *dE = rates + (int64_t)(dim + 1) * n;
    cudaStream_t s = as_stream(stream);
    const CompK K = consts(p);
    for (int k = 0; k < nsteps; ++k) {
        launch_rates(p, st, K, drho, dmom, dE, s);
        k_comp_update<<<grid_for(n, 256), 256, 0, s>>>(st->rho, st->mom, st->E, drho, dmom, dE, n, dim, p->dt);
        SPH_LAUNCH_CHECK(ctx);
    }
    return SPH_OK;
}
