// a12: learned relaxation proposal -- features, a 128-128-128-128-3 GELU MLP on
// BF16 tensor cores (mma.sync m16n8k16, float32 accumulation), its backward pass,
// Adam, and the proposal step that moves particles by the predicted displacement.
//
// One tiled GEMM kernel serves every dense layer of the forward and backward
// passes: C[M x N] = op(A)[M x K] op(B)[K x N] with float32 operands in global
// memory, converted to bfloat16 while staging 64 x 32 tiles into shared memory,
// and an epilogue that adds a bias and applies GELU (storing the pre-activation
// for the backward pass).  Reductions (bias gradients, loss) use a fixed order.
#include <cuda_bf16.h>
#include "common.cuh"
#include "gelu.cuh"
#include "neighbors.cuh"

namespace {

constexpr int NIN = 128, NHID = 128, NOUT = 3, NNEIGH = 32;
// flat parameter layout: W1 (128x128) b1 W2 b2 W3 b3 W4 (3x128) b4
constexpr int64_t OFF_W1 = 0, OFF_B1 = OFF_W1 + NHID * NIN;
constexpr int64_t OFF_W2 = OFF_B1 + NHID, OFF_B2 = OFF_W2 + NHID * NHID;
constexpr int64_t OFF_W3 = OFF_B2 + NHID, OFF_B3 = OFF_W3 + NHID * NHID;
constexpr int64_t OFF_W4 = OFF_B3 + NHID, OFF_B4 = OFF_W4 + NOUT * NHID;
constexpr int64_t NPARAM = OFF_B4 + NOUT;
static_assert(NPARAM == SPH_MLP_NPARAM, "parameter layout");

// ------------------------------------------------------------------ GEMM
constexpr int BM = 64, BN = 64, BK = 32, PAD = 8;
enum { EPI_NONE = 0, EPI_BIAS = 1, EPI_BIAS_GELU = 2 };

__device__ __forceinline__ float gelu_f(float z) { return gelu_as::gelu(z); }
__device__ __forceinline__ float gelu_grad_f(float z) { return gelu_as::gelu_grad(z); }

__device__ __forceinline__ void mma_bf16(float* c, const uint32_t* a, const uint32_t* b) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// C = op(A) op(B) (+ bias, GELU).  A stored [M][K] (aT = 0) or [K][M] (aT = 1);
// B stored [K][N] (bT = 0) or [N][K] (bT = 1).  128 threads, 2 x 2 warps of 32 x 32.
// blockIdx.z selects a slice [z kchunk, (z + 1) kchunk) of K whose product goes to
// C + z * slice_stride (split-K; slices are summed by k_sum_slices).
template <int EPI>
__global__ void __launch_bounds__(128) k_gemm_bf16(int M, int N, int K, const float* __restrict__ A, int lda, int aT,
                                                   const float* __restrict__ B, int ldb, int bT,
                                                   const float* __restrict__ bias, float* __restrict__ C, int ldc,
                                                   float* __restrict__ Zout, int kchunk, int64_t slice_stride) {
    __shared__ __align__(16) __nv_bfloat16 As[BM][BK + PAD];
    __shared__ __align__(16) __nv_bfloat16 Bs[BN][BK + PAD];
    int tid = threadIdx.x;
    int warp = tid >> 5, lane = tid & 31;
    int wm = warp >> 1, wn = warp & 1;
    int gid = lane >> 2, tig = lane & 3;
    int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    float acc[2][4][4];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[a][b][c] = 0.0f;
    const int kb = blockIdx.z * kchunk, ke = min(K, kb + kchunk);
    C += (int64_t)blockIdx.z * slice_stride;
    for (int k0 = kb; k0 < ke; k0 += BK) {
#pragma unroll 4
        for (int r = 0; r < (BM * BK) / 128; ++r) {
            int idx = tid + 128 * r;
            int m, k;
            if (!aT) { m = idx / BK; k = idx % BK; }
            else { k = idx / BM; m = idx % BM; }
            int gm = m0 + m, gk = k0 + k;
            float v = 0.0f;
            if (gm < M && gk < ke) v = aT ? A[(int64_t)gk * lda + gm] : A[(int64_t)gm * lda + gk];
            As[m][k] = __float2bfloat16_rn(v);
        }
#pragma unroll 4
        for (int r = 0; r < (BN * BK) / 128; ++r) {
            int idx = tid + 128 * r;
            int n, k;
            if (bT) { n = idx / BK; k = idx % BK; }
            else { k = idx / BN; n = idx % BN; }
            int gn = n0 + n, gk = k0 + k;
            float v = 0.0f;
            if (gn < N && gk < ke) v = bT ? B[(int64_t)gn * ldb + gk] : B[(int64_t)gk * ldb + gn];
            Bs[n][k] = __float2bfloat16_rn(v);
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; kk += 16) {
            uint32_t af[2][4], bf[4][2];
#pragma unroll
            for (int mi = 0; mi < 2; ++mi) {
                int r0 = wm * 32 + mi * 16 + gid;
                af[mi][0] = *reinterpret_cast<const uint32_t*>(&As[r0][kk + 2 * tig]);
                af[mi][1] = *reinterpret_cast<const uint32_t*>(&As[r0 + 8][kk + 2 * tig]);
                af[mi][2] = *reinterpret_cast<const uint32_t*>(&As[r0][kk + 2 * tig + 8]);
                af[mi][3] = *reinterpret_cast<const uint32_t*>(&As[r0 + 8][kk + 2 * tig + 8]);
            }
#pragma unroll
            for (int ni = 0; ni < 4; ++ni) {
                int c0 = wn * 32 + ni * 8 + gid;
                bf[ni][0] = *reinterpret_cast<const uint32_t*>(&Bs[c0][kk + 2 * tig]);
                bf[ni][1] = *reinterpret_cast<const uint32_t*>(&Bs[c0][kk + 2 * tig + 8]);
            }
#pragma unroll
            for (int mi = 0; mi < 2; ++mi)
#pragma unroll
                for (int ni = 0; ni < 4; ++ni) mma_bf16(acc[mi][ni], af[mi], bf[ni]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int mi = 0; mi < 2; ++mi)
#pragma unroll
        for (int ni = 0; ni < 4; ++ni)
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                int row = m0 + wm * 32 + mi * 16 + gid + (c >= 2 ? 8 : 0);
                int col = n0 + wn * 32 + ni * 8 + 2 * tig + (c & 1);
                if (row < M && col < N) {
                    float v = acc[mi][ni][c];
                    if (EPI != EPI_NONE) v += bias[col];
                    if (EPI == EPI_BIAS_GELU) {
                        Zout[(int64_t)row * ldc + col] = v;
                        C[(int64_t)row * ldc + col] = gelu_f(v);
                    } else {
                        C[(int64_t)row * ldc + col] = v;
                    }
                }
            }
}

}  // namespace

// The tcgen05 form of the GEMM above (mlp_tc.cu): same operands, slices and epilogues.
int sph_gemm_tc(sph_ctx* ctx, int epi, int M, int N, int K, const float* A, int lda, int aT, const float* B, int ldb,
                int bT, const float* bias, float* C, int ldc, float* Z, int kchunk, int slices, int64_t slice_stride,
                cudaStream_t s);

namespace {

// tc != nullptr: the tcgen05 GEMM (the training path); else the mma.sync one (the
// reference forward, sph_mlp_forward).
void gemm(int epi, int M, int N, int K, const float* A, int lda, int aT, const float* B, int ldb, int bT,
          const float* bias, float* C, int ldc, float* Z, cudaStream_t s, sph_ctx* tc = nullptr) {
    if (tc) {
        sph_gemm_tc(tc, epi, M, N, K, A, lda, aT, B, ldb, bT, bias, C, ldc, Z, K, 1, 0, s);
        return;
    }
    dim3 grid((N + BN - 1) / BN, (M + BM - 1) / BM);
    if (epi == EPI_NONE)
        k_gemm_bf16<EPI_NONE><<<grid, 128, 0, s>>>(M, N, K, A, lda, aT, B, ldb, bT, bias, C, ldc, Z, K, 0);
    else if (epi == EPI_BIAS)
        k_gemm_bf16<EPI_BIAS><<<grid, 128, 0, s>>>(M, N, K, A, lda, aT, B, ldb, bT, bias, C, ldc, Z, K, 0);
    else
        k_gemm_bf16<EPI_BIAS_GELU><<<grid, 128, 0, s>>>(M, N, K, A, lda, aT, B, ldb, bT, bias, C, ldc, Z, K, 0);
}

// out[e] = sum over z of parts[z][e], z ascending (a fixed order: deterministic).
__global__ void k_sum_slices(const float* __restrict__ parts, int slices, int64_t count, float* __restrict__ out) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= count) return;
    float acc = 0.0f, comp = 0.0f;
    for (int z = 0; z < slices; ++z) {
        float y = parts[(int64_t)z * count + e] - comp;
        float t = acc + y;
        comp = (t - acc) - y;
        acc = t;
    }
    out[e] = acc - comp;
}

// Weight gradient C[M][N] (ldc = N) = op(A) op(B) over a long K (the batch): the K
// range is cut into slices computed by separate blocks, then summed in order.
void gemm_splitk(int M, int N, int K, const float* A, int lda, int aT, const float* B, int ldb, int bT, float* C,
                 float* scratch, cudaStream_t s, sph_ctx* tc = nullptr) {
    int slices = (K + 255) / 256;
    if (slices > 64) slices = 64;
    // tcgen05: slices of whole 128-row chunks
    const int kq = tc ? 128 : BK;
    int kchunk = ((K + slices - 1) / slices + kq - 1) / kq * kq;
    slices = (K + kchunk - 1) / kchunk;
    if (tc) {
        sph_gemm_tc(tc, EPI_NONE, M, N, K, A, lda, aT, B, ldb, bT, nullptr, scratch, N, nullptr, kchunk, slices,
                    (int64_t)M * N, s);
    } else {
        dim3 grid((N + BN - 1) / BN, (M + BM - 1) / BM, slices);
        k_gemm_bf16<EPI_NONE><<<grid, 128, 0, s>>>(M, N, K, A, lda, aT, B, ldb, bT, nullptr, scratch, N, nullptr,
                                                    kchunk, (int64_t)M * N);
    }
    k_sum_slices<<<grid_for((int64_t)M * N, 256), 256, 0, s>>>(scratch, slices, (int64_t)M * N, C);
}

// Column sums of X[rows][cols] (the bias gradients): per-slice partial sums, then
// the slices summed in order.
__global__ void k_colsum_slices(const float* __restrict__ X, int64_t rows, int cols, int64_t rchunk,
                                float* __restrict__ parts) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= cols) return;
    int64_t r0 = (int64_t)blockIdx.y * rchunk, r1 = r0 + rchunk < rows ? r0 + rchunk : rows;
    float acc = 0.0f, comp = 0.0f;
    for (int64_t r = r0; r < r1; ++r) {
        float y = X[r * cols + c] - comp;
        float t = acc + y;
        comp = (t - acc) - y;
        acc = t;
    }
    parts[(int64_t)blockIdx.y * cols + c] = acc - comp;
}

void colsum(const float* X, int64_t rows, int cols, float* out, float* scratch, cudaStream_t s) {
    int slices = (int)((rows + 63) / 64);
    if (slices > 64) slices = 64;
    int64_t rchunk = (rows + slices - 1) / slices;
    slices = (int)((rows + rchunk - 1) / rchunk);
    dim3 grid((cols + 127) / 128, slices);
    k_colsum_slices<<<grid, 128, 0, s>>>(X, rows, cols, rchunk, scratch);
    k_sum_slices<<<grid_for(cols, 256), 256, 0, s>>>(scratch, slices, cols, out);
}

// ------------------------------------------------------------------ elementwise / reductions
__global__ void k_gelu_backward(const float* __restrict__ dH, const float* __restrict__ Z, float* __restrict__ dZ,
                                int64_t count) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) dZ[i] = dH[i] * gelu_grad_f(Z[i]);
}

// dY = 2 (Y - T) / (3 B); per-block partial sums of (Y - T)^2 in float64.
__global__ void k_mse(const float* __restrict__ Y, const float* __restrict__ T, int64_t count, double inv,
                      float* __restrict__ dY, double* __restrict__ partial) {
    __shared__ double sh[256];
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double e = 0.0;
    if (i < count) {
        float d = Y[i] - T[i];
        dY[i] = (float)(2.0 * inv) * d;
        e = (double)d * (double)d;
    }
    sh[threadIdx.x] = e;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = sh[0];
}

__global__ void k_sum_partial(const double* __restrict__ partial, int nb, double scale, double* __restrict__ out) {
    __shared__ double sh[256];
    double a = 0.0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) a += partial[b];
    sh[threadIdx.x] = a;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = sh[0] * scale;
}

// column sums of X [rows][cols] in fixed row order (bias gradients)

__global__ void k_adam(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                       int64_t count, float lr, float b1, float b2, float eps, float bc1, float bc2) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    float gi = g[i];
    float mi = b1 * m[i] + (1.0f - b1) * gi;
    float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    float mh = mi / bc1, vh = vi / bc2;
    w[i] -= lr * mh / (sqrtf(vh) + eps);
}

// ------------------------------------------------------------------ features
struct FeatSpheres {
    int count;
    double c[SPH_MAX_SPHERES][3];
    double r[SPH_MAX_SPHERES];
};

__device__ __forceinline__ double sdf_union(const FeatSpheres& S, const double* x, double* g) {
    double best = 0.0;
    int arg = 0;
    for (int k = 0; k < S.count; ++k) {
        double dx = x[0] - S.c[k][0], dy = x[1] - S.c[k][1], dz = x[2] - S.c[k][2];
        double d = sqrt(dx * dx + dy * dy + dz * dz) - S.r[k];
        if (k == 0 || d < best) { best = d; arg = k; }
    }
    if (g) {
        double rx = x[0] - S.c[arg][0], ry = x[1] - S.c[arg][1], rz = x[2] - S.c[arg][2];
        double nr = sqrt(rx * rx + ry * ry + rz * rz);
        if (nr > 0.0) { g[0] = rx / nr; g[1] = ry / nr; g[2] = rz / nr; }
        else { g[0] = 1.0; g[1] = 0.0; g[2] = 0.0; }
    }
    return best;
}

// Squared distance of the feature ranking: float64, each operation rounded on its own,
// axes in order.
__device__ __forceinline__ double feat_d2(const double* xi, const double* __restrict__ pos, int64_t n, int j) {
    double d2 = 0.0;
    for (int a = 0; a < 3; ++a) {
        double dx = __dsub_rn(xi[a], pos[a * n + j]);
        double sq = __dmul_rn(dx, dx);
        d2 = a == 0 ? sq : __dadd_rn(d2, sq);
    }
    return d2;
}

// 32 nearest neighbours by (float64 squared distance, j), offsets / h, then phi / h, one
// thread per particle.
__global__ void k_features(const double* __restrict__ pos, int64_t n, const int64_t* __restrict__ row_ptr,
                           const int32_t* __restrict__ col, FeatSpheres S, double inv_h, float* __restrict__ feats) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double xi[3] = {pos[i], pos[n + i], pos[2 * n + i]};
    double bd[NNEIGH];
    int bj[NNEIGH];
    int cnt = 0;
    for (int64_t p = row_ptr[i], e = row_ptr[i + 1]; p < e; ++p) {
        int j = col[p];
        const double d2 = feat_d2(xi, pos, n, j);
        // insert into the sorted list of the best NNEIGH (key: d2, then j)
        int k = cnt < NNEIGH ? cnt : NNEIGH;
        if (k == NNEIGH && !(d2 < bd[NNEIGH - 1] || (d2 == bd[NNEIGH - 1] && j < bj[NNEIGH - 1]))) continue;
        if (k == NNEIGH) k = NNEIGH - 1;
        while (k > 0 && (d2 < bd[k - 1] || (d2 == bd[k - 1] && j < bj[k - 1]))) {
            bd[k] = bd[k - 1];
            bj[k] = bj[k - 1];
            --k;
        }
        bd[k] = d2;
        bj[k] = j;
        if (cnt < NNEIGH) ++cnt;
    }
    float* f = feats + i * NIN;
    for (int k = 0; k < NNEIGH; ++k) {
        if (k < cnt) {
            int j = bj[k];
            for (int a = 0; a < 3; ++a) f[3 * k + a] = (float)((pos[a * n + j] - xi[a]) * inv_h);
        } else {
            f[3 * k] = f[3 * k + 1] = f[3 * k + 2] = 0.0f;
        }
    }
    f[3 * NNEIGH] = (float)(sdf_union(S, xi, nullptr) * inv_h);
    for (int k = 3 * NNEIGH + 1; k < NIN; ++k) f[k] = 0.0f;
}

void launch_features(const double* pos, int64_t n, const int64_t* rp, const int32_t* cl, const FeatSpheres& S,
                     double inv_h, float* feats, cudaStream_t s) {
    k_features<<<grid_for(n, 128), 128, 0, s>>>(pos, n, rp, cl, S, inv_h, feats);
}

// x += h * dx_pred, then projection to phi <= -dp/2
__global__ void k_apply_proposal(double* __restrict__ pos, int64_t n, const float* __restrict__ out, FeatSpheres S,
                                 double h, double dp) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double x[3];
    for (int a = 0; a < 3; ++a) x[a] = pos[a * n + i] + h * (double)out[i * NOUT + a];
    double g[3];
    double phi = sdf_union(S, x, g);
    if (phi > -0.5 * dp) {
        double sh = phi + 0.5 * dp;
        for (int a = 0; a < 3; ++a) x[a] -= sh * g[a];
    }
    for (int a = 0; a < 3; ++a) pos[a * n + i] = x[a];
}

// ------------------------------------------------------------------ host helpers
struct Act {
    float *Z1, *H1, *Z2, *H2, *Z3, *H3, *Y;
};

int forward_chunk(const float* P, const float* X, int64_t rows, Act& a, cudaStream_t s, sph_ctx* tc = nullptr) {
    int M = (int)rows;
    gemm(EPI_BIAS_GELU, M, NHID, NIN, X, NIN, 0, P + OFF_W1, NIN, 1, P + OFF_B1, a.H1, NHID, a.Z1, s, tc);
    gemm(EPI_BIAS_GELU, M, NHID, NHID, a.H1, NHID, 0, P + OFF_W2, NHID, 1, P + OFF_B2, a.H2, NHID, a.Z2, s, tc);
    gemm(EPI_BIAS_GELU, M, NHID, NHID, a.H2, NHID, 0, P + OFF_W3, NHID, 1, P + OFF_B3, a.H3, NHID, a.Z3, s, tc);
    gemm(EPI_BIAS, M, NOUT, NHID, a.H3, NHID, 0, P + OFF_W4, NHID, 1, P + OFF_B4, a.Y, NOUT, nullptr, s, tc);
    return cudaGetLastError() == cudaSuccess ? SPH_OK : SPH_ERR_CUDA;
}

int alloc_act(sph_ctx* ctx, int64_t rows, Act& a) {
    int st = SPH_OK;
    size_t hb = (size_t)rows * NHID * 4;
    float* base = (float*)sph_scratch(ctx, S_MISC1, 6 * hb + (size_t)rows * 4 * 4 + 256, &st);
    if (st) return st;
    a.Z1 = base;
    a.H1 = a.Z1 + rows * NHID;
    a.Z2 = a.H1 + rows * NHID;
    a.H2 = a.Z2 + rows * NHID;
    a.Z3 = a.H2 + rows * NHID;
    a.H3 = a.Z3 + rows * NHID;
    a.Y = a.H3 + rows * NHID;
    return SPH_OK;
}

constexpr int64_t kForwardChunk = 1 << 18;

FeatSpheres feat_spheres(const sph_relax_params* p) {
    FeatSpheres S;
    S.count = p->n_spheres;
    for (int k = 0; k < SPH_MAX_SPHERES; ++k) {
        for (int c = 0; c < 3; ++c) S.c[k][c] = k < S.count ? p->spheres[4 * k + c] : 0.0;
        S.r[k] = k < S.count ? p->spheres[4 * k + 3] : 0.0;
    }
    return S;
}

int mlp_grad_impl(sph_ctx* ctx, const float* P, const float* X, const float* T, int64_t B, float* grad,
                  double* loss_host, cudaStream_t s) {
    Act a;
    int st = alloc_act(ctx, B, a);
    if (st) return st;
    // the training path's GEMMs on tcgen05 (tensor-memory accumulators)
    st = forward_chunk(P, X, B, a, s, ctx);
    if (st) return st;
    int nb = (int)grid_for(B * NOUT, 256);
    float* dY = (float*)sph_scratch(ctx, S_MISC0, (size_t)B * NOUT * 4 + (size_t)B * NHID * 8 + 256, &st);
    double* partial = (double*)sph_scratch(ctx, S_RED_PARTIAL, (size_t)nb * 8 + 64, &st);
    if (st) return st;
    float* dH = dY + ((B * NOUT + 63) / 64) * 64;
    float* dZ = dH + B * NHID;
    double* loss_d = partial + nb;
    double inv = 1.0 / ((double)B * NOUT);
    k_mse<<<nb, 256, 0, s>>>(a.Y, T, B * NOUT, inv, dY, partial);
    k_sum_partial<<<1, 256, 0, s>>>(partial, nb, inv, loss_d);
    // split-K partials of the weight gradients (64 slices of at most 128 x 128)
    float* parts = (float*)sph_scratch(ctx, S_MLP_PARTS, (size_t)64 * NHID * NHID * 4 + 256, &st);
    if (st) return st;
    // layer 4
    gemm_splitk(NOUT, NHID, (int)B, dY, NOUT, 1, a.H3, NHID, 0, grad + OFF_W4, parts, s, ctx);
    colsum(dY, B, NOUT, grad + OFF_B4, parts, s);
    gemm(EPI_NONE, (int)B, NHID, NOUT, dY, NOUT, 0, P + OFF_W4, NHID, 0, nullptr, dH, NHID, nullptr, s, ctx);
    const float* Zs[3] = {a.Z1, a.Z2, a.Z3};
    const float* Hin[3] = {X, a.H1, a.H2};
    const int64_t offW[3] = {OFF_W1, OFF_W2, OFF_W3}, offB[3] = {OFF_B1, OFF_B2, OFF_B3};
    const int nin[3] = {NIN, NHID, NHID};
    for (int l = 2; l >= 0; --l) {
        k_gelu_backward<<<grid_for(B * NHID, 256), 256, 0, s>>>(dH, Zs[l], dZ, B * NHID);
        gemm_splitk(NHID, nin[l], (int)B, dZ, NHID, 1, Hin[l], nin[l], 0, grad + offW[l], parts, s, ctx);
        colsum(dZ, B, NHID, grad + offB[l], parts, s);
        if (l > 0)
            gemm(EPI_NONE, (int)B, nin[l], NHID, dZ, NHID, 0, P + offW[l], nin[l], 0, nullptr, dH, nin[l], nullptr, s,
                 ctx);
    }
    SPH_LAUNCH_CHECK(ctx);
    if (loss_host) {
        double* hp = (double*)ctx->pinned;
        SPH_CUDA(ctx, cudaMemcpyAsync(hp + 40, loss_d, 8, cudaMemcpyDeviceToHost, s));
        SPH_CUDA(ctx, cudaStreamSynchronize(s));
        *loss_host = hp[40];
        // the tcgen05 GEMMs' bounded waits: reported with the loss, when the call syncs
        int r = sph_take_status(ctx, s);
        if (r) return r;
    }
    return SPH_OK;
}

int check_relax_like(const sph_relax_params* p) {
    if (!p) return SPH_ERR_ARG;
    int s = sph_check_domain(&p->dom);
    if (s) return s;
    if (p->dom.dim != 3 || p->n_spheres < 1 || p->n_spheres > SPH_MAX_SPHERES) return SPH_ERR_ARG;
    return SPH_OK;
}

// LG-support neighbour lists of the current positions into context scratch.
int lists_for(sph_ctx* ctx, const sph_relax_params* p, const double* pos, cudaStream_t s, int64_t** rp, int32_t** cl) {
    sph_domain dom = p->dom;
    dom.kappa = 2.0;
    int64_t n = dom.n;
    CellList c;
    int st = sph_build_cells(ctx, &dom, pos, s, &c);
    if (st) return st;
    int32_t* row_len = (int32_t*)sph_scratch(ctx, S_ROW_LEN, (size_t)(n + 1) * 4, &st);
    int64_t* row_ptr = (int64_t*)sph_scratch(ctx, S_RELAX_ROWPTR, (size_t)(n + 1) * 8, &st);
    if (st) return st;
    st = sph_count_neighbors(ctx, c, pos, n, c.grid.rc2, row_len, s);
    if (st) return st;
    st = sph_exclusive_scan_i64(ctx, row_len, row_ptr, n, s);
    if (st) return st;
    int64_t* hp = (int64_t*)ctx->pinned;
    SPH_CUDA(ctx, cudaMemcpyAsync(hp + 8, row_ptr + n, 8, cudaMemcpyDeviceToHost, s));
    SPH_CUDA(ctx, cudaMemcpyAsync((int*)ctx->pinned, ctx->flags, FLAG_COUNT * sizeof(int), cudaMemcpyDeviceToHost, s));
    SPH_CUDA(ctx, cudaMemsetAsync(ctx->flags, 0, FLAG_COUNT * sizeof(int), s));
    SPH_CUDA(ctx, cudaStreamSynchronize(s));
    if (((int*)ctx->pinned)[FLAG_BAD_INPUT]) return SPH_ERR_ARG;
    int64_t nnz = hp[8];
    int32_t* col = (int32_t*)sph_scratch(ctx, S_RELAX_COL, (size_t)nnz * 4 + 16, &st);
    if (st) return st;
    st = sph_fill_neighbors(ctx, c, pos, n, c.grid.rc2, row_ptr, col, nnz, s);
    *rp = row_ptr;
    *cl = col;
    return st;
}

}  // namespace

extern "C" int sph_mlp_forward(sph_ctx* ctx, const float* params, const float* feats, float* out, int64_t n,
                               void* stream) {
    if (!ctx || n < 0) return SPH_ERR_ARG;
    if (n == 0) return SPH_OK;
    if (!params || !feats || !out) return SPH_ERR_ARG;
    cudaStream_t s = as_stream(stream);
    int64_t chunk = n < kForwardChunk ? n : kForwardChunk;
    Act a;
    int st = alloc_act(ctx, chunk, a);
    if (st) return st;
    for (int64_t r0 = 0; r0 < n; r0 += chunk) {
        int64_t rows = n - r0 < chunk ? n - r0 : chunk;
        a.Y = out + r0 * NOUT;
        st = forward_chunk(params, feats + r0 * NIN, rows, a, s);
        if (st) { ctx->last_cuda_error = (int)cudaGetLastError(); return st; }
    }
    return SPH_OK;
}

extern "C" int sph_mlp_grad(sph_ctx* ctx, const float* params, const float* feats, const float* target, int64_t b,
                            float* grad, double* loss_host, void* stream) {
    if (!ctx || b <= 0 || b > (1 << 22) || !params || !feats || !target || !grad) return SPH_ERR_ARG;
    return mlp_grad_impl(ctx, params, feats, target, b, grad, loss_host, as_stream(stream));
}

extern "C" int sph_mlp_train_step(sph_ctx* ctx, float* params, float* adam_m, float* adam_v, int64_t step, double lr,
                                  const float* feats, const float* target, int64_t b, double* loss_host,
                                  void* stream) {
    if (!ctx || b <= 0 || b > (1 << 22) || step < 1 || !(lr > 0.0)) return SPH_ERR_ARG;
    if (!params || !adam_m || !adam_v || !feats || !target) return SPH_ERR_ARG;
    cudaStream_t s = as_stream(stream);
    int st = SPH_OK;
    float* grad = (float*)sph_scratch(ctx, S_MISC2, NPARAM * 4 + 256, &st);
    if (st) return st;
    st = mlp_grad_impl(ctx, params, feats, target, b, grad, loss_host, s);
    if (st) return st;
    const double b1 = 0.9, b2 = 0.999;
    float bc1 = (float)(1.0 - pow(b1, (double)step)), bc2 = (float)(1.0 - pow(b2, (double)step));
    k_adam<<<grid_for(NPARAM, 256), 256, 0, s>>>(params, grad, adam_m, adam_v, NPARAM, (float)lr, (float)b1, (float)b2,
                                                 1e-8f, bc1, bc2);
    SPH_LAUNCH_CHECK(ctx);
    return SPH_OK;
}

extern "C" int sph_mlp_features(sph_ctx* ctx, const sph_relax_params* p, const double* pos, float* feats,
                                void* stream) {
    if (!ctx) return SPH_ERR_ARG;
    int st = check_relax_like(p);
    if (st) return st;
    int64_t n = p->dom.n;
    if (n == 0) return SPH_OK;
    if (!pos || !feats) return SPH_ERR_ARG;
    cudaStream_t s = as_stream(stream);
    int64_t* rp = nullptr;
    int32_t* cl = nullptr;
    st = lists_for(ctx, p, pos, s, &rp, &cl);
    if (st) return st;
    launch_features(pos, n, rp, cl, feat_spheres(p), 1.0 / p->dom.h, feats, s);
    SPH_LAUNCH_CHECK(ctx);
    return SPH_OK;
}

extern "C" int sph_relax_propose(sph_ctx* ctx, const sph_relax_params* p, const float* params, double* pos,
                                 void* stream) {
    if (!ctx || !params) return SPH_ERR_ARG;
    int st = check_relax_like(p);
    if (st) return st;
    int64_t n = p->dom.n;
    if (n == 0) return SPH_OK;
    if (!pos) return SPH_ERR_ARG;
    cudaStream_t s = as_stream(stream);
    int64_t* rp = nullptr;
    int32_t* cl = nullptr;
    st = lists_for(ctx, p, pos, s, &rp, &cl);
    if (st) return st;
    float* buf = (float*)sph_scratch(ctx, S_MISC3, (size_t)n * (NIN + NOUT) * 4 + 256, &st);
    if (st) return st;
    float* feats = buf;
    float* out = buf + n * NIN;
    FeatSpheres S = feat_spheres(p);
    launch_features(pos, n, rp, cl, S, 1.0 / p->dom.h, feats, s);
    SPH_LAUNCH_CHECK(ctx);
    // the fused tensor-core forward (same network as sph_mlp_forward)
    st = sph_mlp_forward_tc(ctx, params, feats, out, n, stream);
    if (st) return st;
    k_apply_proposal<<<grid_for(n, 256), 256, 0, s>>>(pos, n, out, S, p->dom.h, p->dp);
    SPH_LAUNCH_CHECK(ctx);
    return SPH_OK;
}
