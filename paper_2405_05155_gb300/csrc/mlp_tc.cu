// a12: fused forward of the 128-128-128-128-3 GELU MLP on the fifth-generation
// tensor cores (tcgen05, accumulators in tensor memory).
//
// One persistent block per SM keeps the four layers' weights in shared memory as
// bfloat16 for the whole launch.  Its sixteen warps form two independent groups
// of eight, each walking its own tiles of 128 rows with its own activation
// buffer, mbarrier and 128 columns of tensor memory, so that one group's MMAs run
// while the other group's warps evaluate GELU.  Per tile and layer, one thread of
// the group issues eight tcgen05.mma (M = 128, N = 128, K = 16; A = the tile's
// activations, B = the layer's weights, both bfloat16 from shared memory, float32
// accumulation in tensor memory) and commits them to the group's mbarrier; the
// group's warps read the accumulator back with tcgen05.ld (four lane quarters x
// two 64-column halves), add the bias, apply GELU and write the next layer's
// bfloat16 operand into shared memory.  The last layer (3 outputs) runs with
// N = 16 over zero-padded weights.  The activations never leave the SM; global
// memory sees the float32 features once and the outputs.
//
// Operands use the no-swizzle K-major layout of 8 x 16-byte core matrices:
// element (r, k) of a [rows x 128] bfloat16 matrix lives at byte
// ((r / 8) * 16 + k / 8) * 128 + (r % 8) * 16 + (k % 8) * 2, so neighbouring core
// matrices along K are 128 bytes apart (leading byte offset) and neighbouring
// 8-row groups 2048 bytes apart (stride byte offset).
#include <cuda_bf16.h>
#include "common.cuh"
#include "gelu.cuh"
#include "async.cuh"

namespace {

constexpr int kRows = 128;      // rows per tile: the MMA's M
constexpr int kWidth = 128;     // hidden width: N of layers 1-3 and K of every layer
constexpr int kOut = 3;
constexpr int kOutPad = 16;     // N of the last layer (smallest N for M = 128)
constexpr int kThreads = 512;
constexpr int kGroups = 2;
constexpr int kGroupThreads = kThreads / kGroups;
constexpr int kTmemCols = 128 * kGroups;
constexpr uint32_t kPolls = 1u << 20;

// flat parameter layout: W1 (128x128, [out][in]) b1 W2 b2 W3 b3 W4 (3x128) b4
constexpr int64_t OFF_W1 = 0, OFF_B1 = OFF_W1 + kWidth * kWidth;
constexpr int64_t OFF_W2 = OFF_B1 + kWidth, OFF_B2 = OFF_W2 + kWidth * kWidth;
constexpr int64_t OFF_W3 = OFF_B2 + kWidth, OFF_B3 = OFF_W3 + kWidth * kWidth;
constexpr int64_t OFF_W4 = OFF_B3 + kWidth, OFF_B4 = OFF_W4 + kOut * kWidth;
static_assert(OFF_B4 + kOut == SPH_MLP_NPARAM, "parameter layout");

constexpr uint32_t kMatBytes = kRows * kWidth * 2;        // 32 KB: one 128 x 128 bfloat16 operand
constexpr uint32_t kW4Bytes = kOutPad * kWidth * 2;       // 4 KB
// shared memory: W1 | W2 | W3 | W4 | activations (one per group) | biases |
// barriers (one per group), tensor-memory base
constexpr uint32_t kOffA = 3 * kMatBytes + kW4Bytes;
constexpr uint32_t kOffBias = kOffA + kGroups * kMatBytes;
constexpr uint32_t kOffBar = kOffBias + (3 * kWidth + kOutPad) * 4;
constexpr uint32_t kSmemBytes = kOffBar + 8 * kGroups + 16;

__device__ __forceinline__ uint32_t cm_offset(int r, int k) {
    return (uint32_t)((((r >> 3) * (kWidth / 8) + (k >> 3)) << 7) + ((r & 7) << 4) + ((k & 7) << 1));
}

// tcgen05 shared-memory matrix descriptor: start address, leading and stride byte
// offsets (all >> 4), descriptor version 1 (bits 46-48), no swizzle.
__device__ __forceinline__ uint64_t mat_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// Instruction descriptor of kind::f16: float32 D, bfloat16 A and B, both K-major,
// N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t inst_desc(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Block barrier that orders shared-memory writes before the tensor cores read them
// and tensor-memory reads before the next MMA overwrites them.
__device__ __forceinline__ void tc_sync() {
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
}

// The same for one group's warps (named barrier g + 1 of kGroupThreads threads).
__device__ __forceinline__ void group_sync(int g) {
    fence_async_smem();
    tc_fence_before();
    asm volatile("bar.sync %0, %1;" ::"r"(g + 1), "r"(kGroupThreads) : "memory");
    tc_fence_after();
}

// Group barrier returning whether any of the group's threads passed p = true.
__device__ __forceinline__ bool group_sync_or(int g, bool p) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred q, o;\n\t"
        "setp.ne.u32 q, %2, 0;\n\t"
        "bar.red.or.pred o, %1, %3, q;\n\t"
        "selp.u32 %0, 1, 0, o;\n\t}"
        : "=r"(r)
        : "r"(g + 1), "r"((uint32_t)p), "r"(kGroupThreads)
        : "memory");
    return r != 0;
}

// 32 consecutive float32 columns of the warp's lane quarter (one row per thread).
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int k = 0; k < 32; ++k) v[k] = __uint_as_float(r[k]);
}

__device__ __forceinline__ float gelu(float z) { return gelu_as::gelu(z); }

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
    __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t*>(&h);
}

// Eight consecutive values (k..k+7 of row r) into the core-matrix operand.
__device__ __forceinline__ void store8(unsigned char* mat, int r, int k, const float* v) {
    uint4 q = make_uint4(pack_bf16(v[0], v[1]), pack_bf16(v[2], v[3]), pack_bf16(v[4], v[5]), pack_bf16(v[6], v[7]));
    *reinterpret_cast<uint4*>(mat + cm_offset(r, k)) = q;
}

__global__ void __launch_bounds__(kThreads, 1) k_mlp_forward_tc(const float* __restrict__ P,
                                                                const float* __restrict__ X,
                                                                float* __restrict__ Y, int64_t n,
                                                                int* __restrict__ flags) {
    extern __shared__ __align__(1024) unsigned char sm[];
    unsigned char* W[3] = {sm, sm + kMatBytes, sm + 2 * kMatBytes};
    unsigned char* W4 = sm + 3 * kMatBytes;
    float* bias = reinterpret_cast<float*>(sm + kOffBias);
    uint64_t* bars = reinterpret_cast<uint64_t*>(sm + kOffBar);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(sm + kOffBar + 8 * kGroups);
    const int tid = threadIdx.x, warp = tid >> 5;

    // weights and biases into shared memory, once
    const int64_t offW[3] = {OFF_W1, OFF_W2, OFF_W3}, offB[3] = {OFF_B1, OFF_B2, OFF_B3};
    for (int q = tid; q < 3 * kWidth * (kWidth / 8); q += kThreads) {
        int l = q / (kWidth * (kWidth / 8)), rem = q % (kWidth * (kWidth / 8));
        int o = rem / (kWidth / 8), k = (rem % (kWidth / 8)) * 8;
        float v[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) v[e] = P[offW[l] + (int64_t)o * kWidth + k + e];
        store8(W[l], o, k, v);
    }
    for (int q = tid; q < kOutPad * (kWidth / 8); q += kThreads) {
        int o = q / (kWidth / 8), k = (q % (kWidth / 8)) * 8;
        float v[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) v[e] = o < kOut ? P[OFF_W4 + (int64_t)o * kWidth + k + e] : 0.0f;
        store8(W4, o, k, v);
    }
    for (int q = tid; q < 3 * kWidth; q += kThreads) bias[q] = P[offB[q / kWidth] + q % kWidth];
    if (tid < kOutPad) bias[3 * kWidth + tid] = tid < kOut ? P[OFF_B4 + tid] : 0.0f;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int g = 0; g < kGroups; ++g) mbar_init(&bars[g], 1);
        mbar_fence_init();
    }
    tc_sync();
    // group g: warps 8g .. 8g + 7, its own tiles, operand buffer, barrier and tensor columns
    const int g = warp / (kGroupThreads / 32), gtid = tid - g * kGroupThreads, gwarp = warp % (kGroupThreads / 32);
    unsigned char* A = sm + kOffA + g * kMatBytes;
    uint64_t* bar = &bars[g];
    const uint32_t tmem = *tmem_slot + (uint32_t)(g * 128);
    const uint32_t sW[3] = {smem_u32(W[0]), smem_u32(W[1]), smem_u32(W[2])};
    const uint32_t sW4 = smem_u32(W4), sA = smem_u32(A);
    // epilogue mapping: warp w of the group reads lane quarter (w % 4), columns 64 (w / 4) .. + 63
    const int quarter = gwarp & 3, chalf = gwarp >> 2;
    const int row = quarter * 32 + (gtid & 31);
    const uint32_t trow = tmem + ((uint32_t)(quarter * 32) << 16);
    uint32_t phase = 0;
    bool ok = true;
    const int64_t tstride = (int64_t)gridDim.x * kGroups;
    for (int64_t tile = (int64_t)blockIdx.x * kGroups + g; tile * kRows < n; tile += tstride) {
        // features (float32) -> bfloat16 operand; rows past n are zero
        {
            const int r = gtid >> 1, k0 = (gtid & 1) * 64;
            const int64_t gr = tile * kRows + r;
            const float4* src = reinterpret_cast<const float4*>(X + gr * kWidth + k0);
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                float v[8];
                if (gr < n) {
                    float4 a = __ldg(src + 2 * c), b = __ldg(src + 2 * c + 1);
                    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w; v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
                } else {
#pragma unroll
                    for (int e = 0; e < 8; ++e) v[e] = 0.0f;
                }
                store8(A, r, k0 + 8 * c, v);
            }
        }
        group_sync(g);
        for (int l = 0; l < 4 && ok; ++l) {
            if (gtid == 0) {
                const uint32_t idesc = l < 3 ? inst_desc(kRows, kWidth) : inst_desc(kRows, kOutPad);
                const uint32_t sB = l < 3 ? sW[l] : sW4;
#pragma unroll
                for (int kk = 0; kk < kWidth / 16; ++kk)
                    mma_bf16(tmem, mat_desc(sA + 256 * kk, 128, 2048), mat_desc(sB + 256 * kk, 128, 2048), idesc,
                             kk > 0);
                mma_commit(bar);
            }
            const bool late = !mbar_wait_bounded(bar, phase, kPolls);
            phase ^= 1u;
            if (group_sync_or(g, late)) {
                ok = false;
                if (gtid == 0) atomicExch(&flags[FLAG_TIMEOUT], 1);
                break;
            }
            tc_fence_after();
            if (l < 3) {
                const float* b = bias + l * kWidth;
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int c0 = chalf * 64 + h * 32;
                    float v[32];
                    tmem_ld32(trow + (uint32_t)c0, v);
                    // + bias and GELU two columns at a time (the bias, in shared memory, read as float4)
#pragma unroll
                    for (int c = 0; c < 32; c += 4) {
                        const float4 bb = *reinterpret_cast<const float4*>(b + c0 + c);
                        const float2 z0 = __fadd2_rn(make_float2(v[c], v[c + 1]), make_float2(bb.x, bb.y));
                        const float2 z1 = __fadd2_rn(make_float2(v[c + 2], v[c + 3]), make_float2(bb.z, bb.w));
                        const float2 g0 = gelu_as::gelu2(z0), g1 = gelu_as::gelu2(z1);
                        v[c] = g0.x;
                        v[c + 1] = g0.y;
                        v[c + 2] = g1.x;
                        v[c + 3] = g1.y;
                    }
#pragma unroll
                    for (int c = 0; c < 4; ++c) store8(A, row, c0 + 8 * c, v + 8 * c);
                }
            } else if (chalf == 0) {
                float v[32];
                tmem_ld32(trow, v);
                const int64_t gr = tile * kRows + row;
                if (gr < n) {
#pragma unroll
                    for (int c = 0; c < kOut; ++c) Y[gr * kOut + c] = v[c] + bias[3 * kWidth + c];
                }
            }
            group_sync(g);
        }
        if (!ok) break;
    }
    tc_sync();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
}

// ---------------------------------------------------------------- training GEMM
// C = op(A) op(B) on tcgen05 for the training path (the dense layers of the forward, the
// backward's products with the weights and the weight gradients): one block computes a
// 128 x BNT tile of C (BNT = 32, or 16 for the 3-output layer), over the K range of its
// slice in chunks of 128.  A is stored [M][K] (aT = 0) or [K][M] (aT = 1), B [K][N] (bT = 0)
// or [N][K] (bT = 1), both float32 in global memory; the loader converts them to bfloat16 and
// writes both operands K-major into the core-matrix layout of the fused forward (a
// transpose is a strided read, never a different descriptor), zero beyond M, N and the
// slice.  One thread issues 8 tcgen05.mma (K = 16) per chunk into 128 columns of tensor
// memory; the 4 warps read the accumulator back (a lane quarter each) and apply the
// epilogue: + bias, and GELU keeping the pre-activation in Zout.  Slice z of a split K
// writes C + z * slice_stride.  A bounded mbarrier wait that expires sets the timeout flag
// and the block writes nothing.
constexpr int kGemmThreads = 128;

__device__ __forceinline__ float tc_load(const float* __restrict__ X, int ld, int t, int r, int k, int R, int ke) {
    // element (r, k) of the operand read as [rows][K]: X[r][k] (t = 0) or X[k][r] (t = 1)
    if (r >= R || k >= ke) return 0.0f;
    return t ? X[(int64_t)k * ld + r] : X[(int64_t)r * ld + k];
}

// rows x 128 operand chunk (K range [k0, k0 + 128) of [0, ke)) into the core-matrix layout.
__device__ __forceinline__ void tc_stage(unsigned char* mat, int rows, const float* __restrict__ X, int ld, int t,
                                         int r0, int R, int k0, int ke) {
    const int groups = rows * (kWidth / 8);
    for (int q = threadIdx.x; q < groups; q += kGemmThreads) {
        // t = 0: consecutive threads take consecutive 8-column groups of a row (contiguous
        // reads along K); t = 1: consecutive threads take consecutive rows (contiguous reads
        // along the rows for each k)
        const int r = t ? q % rows : q / (kWidth / 8);
        const int kg = t ? q / rows : q % (kWidth / 8);
        float v[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) v[e] = tc_load(X, ld, t, r0 + r, k0 + 8 * kg + e, R, ke);
        store8(mat, r, 8 * kg, v);
    }
}

template <int EPI, int BNT>
__global__ void __launch_bounds__(kGemmThreads, 1) k_gemm_tc(int M, int N, int K, const float* __restrict__ A,
                                                              int lda, int aT, const float* __restrict__ B, int ldb,
                                                              int bT, const float* __restrict__ bias,
                                                              float* __restrict__ C, int ldc, float* __restrict__ Zout,
                                                              int kchunk, int64_t slice_stride, int* __restrict__ flags) {
    extern __shared__ __align__(1024) unsigned char sm[];
    unsigned char* As = sm;                         // 128 x 128 bfloat16
    unsigned char* Bs = sm + kMatBytes;             // BNT x 128 bfloat16
    uint64_t* bar = reinterpret_cast<uint64_t*>(sm + kMatBytes + (uint32_t)BNT * kWidth * 2);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bar + 1);
    const int tid = threadIdx.x, warp = tid >> 5;
    const int m0 = blockIdx.y * kRows, n0 = blockIdx.x * BNT;
    const int kb = blockIdx.z * kchunk, ke = min(K, kb + kchunk);
    // tensor-memory columns: BNT, at least 32 (the allocation unit)
    constexpr uint32_t kCols = BNT < 32 ? 32u : (uint32_t)BNT;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(kCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        mbar_init(bar, 1);
        mbar_fence_init();
    }
    tc_sync();
    const uint32_t tmem = *tmem_slot;
    const uint32_t sA = smem_u32(As), sB = smem_u32(Bs);
    constexpr uint32_t idesc = inst_desc(kRows, BNT);
    uint32_t phase = 0;
    bool ok = true;
    for (int k0 = kb; k0 < ke && ok; k0 += kWidth) {
        tc_stage(As, kRows, A, lda, aT, m0, M, k0, ke);
        tc_stage(Bs, BNT, B, ldb, bT ? 0 : 1, n0, N, k0, ke);
        tc_sync();
        if (tid == 0) {
#pragma unroll
            for (int kk = 0; kk < kWidth / 16; ++kk)
                mma_bf16(tmem, mat_desc(sA + 256 * kk, 128, 2048), mat_desc(sB + 256 * kk, 128, 2048), idesc,
                         (k0 > kb || kk > 0) ? 1u : 0u);
            mma_commit(bar);
        }
        const bool late = !mbar_wait_bounded(bar, phase, kPolls);
        phase ^= 1u;
        if (__syncthreads_or(late)) {
            ok = false;
            if (tid == 0) atomicExch(&flags[FLAG_TIMEOUT], 1);
        }
        tc_fence_after();
    }
    if (ok && kb < ke) {
        // warp w: rows 32 w .. 32 w + 31 of the tile, one per lane
        const int row = warp * 32 + (tid & 31);
        const int gm = m0 + row;
        const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
        float* Cz = C + (int64_t)blockIdx.z * slice_stride;
#pragma unroll 1
        for (int c0 = 0; c0 < BNT; c0 += 32) {
            float v[32];
            tmem_ld32(trow + (uint32_t)c0, v);
            if (gm < M) {
#pragma unroll
                for (int c = 0; c < 32; ++c) {
                    const int gn = n0 + c0 + c;
                    if (c0 + c < BNT && gn < N) {
                        float x = v[c];
                        if (EPI != 0) x += bias[gn];
                        if (EPI == 2) {
                            Zout[(int64_t)gm * ldc + gn] = x;
                            x = gelu(x);
                        }
                        Cz[(int64_t)gm * ldc + gn] = x;
                    }
                }
            }
        }
    }
    tc_sync();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kCols) : "memory");
}

}  // namespace

// Forward of the MLP on tcgen05 (see sph.h).
extern "C" int sph_mlp_forward_tc(sph_ctx* ctx, const float* params, const float* feats, float* out, int64_t n,
                                  void* stream) {
    if (!ctx || n < 0) return SPH_ERR_ARG;
    if (n == 0) return SPH_OK;
    if (!params || !feats || !out) return SPH_ERR_ARG;
    if (((uintptr_t)feats & 15u)) return SPH_ERR_ARG;
    cudaStream_t s = as_stream(stream);
    sph_allow_dynamic_smem((const void*)k_mlp_forward_tc);
    int64_t pairs = ((n + kRows - 1) / kRows + kGroups - 1) / kGroups;   // tiles per block and round
    int grid = (int)(pairs < ctx->num_sms ? pairs : ctx->num_sms);
    ctx->waits_pending = true;
    k_mlp_forward_tc<<<grid, kThreads, kSmemBytes, s>>>(params, feats, out, n, ctx->flags);
    SPH_LAUNCH_CHECK(ctx);
    return SPH_OK;
}

// The training GEMM on tcgen05 (declared in mlp.cu's dispatch): epi 0 none, 1 bias, 2 bias
// and GELU; K cut into `slices` slices of kchunk.
int sph_gemm_tc(sph_ctx* ctx, int epi, int M, int N, int K, const float* A, int lda, int aT, const float* B, int ldb,
                int bT, const float* bias, float* C, int ldc, float* Z, int kchunk, int slices, int64_t slice_stride,
                cudaStream_t s) {
    // 128 x 32 tiles: a batch of 4096 rows and 128 outputs makes 128 blocks (the K loop per
    // block is then short; more blocks hide the operand staging)
    const int bnt = N <= 16 ? 16 : 32;
    dim3 grid((unsigned)((N + bnt - 1) / bnt), (unsigned)((M + kRows - 1) / kRows), (unsigned)slices);
    const size_t smem = kMatBytes + (size_t)bnt * kWidth * 2 + 64;
    ctx->waits_pending = true;
#define SPH_GEMM_TC(E, BN)                                                                                 \
    do {                                                                                                   \
        sph_allow_dynamic_smem((const void*)k_gemm_tc<E, BN>);                                             \
        k_gemm_tc<E, BN><<<grid, kGemmThreads, smem, s>>>(M, N, K, A, lda, aT, B, ldb, bT, bias, C, ldc, Z, \
                                                          kchunk, slice_stride, ctx->flags);               \
    } while (0)
    if (bnt == 16) {
        if (epi == 0) SPH_GEMM_TC(0, 16);
        else if (epi == 1) SPH_GEMM_TC(1, 16);
        else SPH_GEMM_TC(2, 16);
    } else {
        if (epi == 0) SPH_GEMM_TC(0, 32);
        else if (epi == 1) SPH_GEMM_TC(1, 32);
        else SPH_GEMM_TC(2, 32);
    }
#undef SPH_GEMM_TC
    return cudaGetLastError() == cudaSuccess ? SPH_OK : SPH_ERR_CUDA;
}
