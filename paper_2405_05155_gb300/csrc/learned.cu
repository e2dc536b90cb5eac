// a12 driven from the C side: the learned relaxation loop, its training data and its
// minibatch training (the proposal is not in the paper; the relaxation it serves and the
// residual that judges it are Sec. 2.3.2-2.3.3).
//
//   sph_relax_samples  plain Laguerre-Gauss trajectory snapshots: features at x^t and
//                      targets (x^{t+every} - x^t)/h, every `every` steps;
//   sph_mlp_train      Adam steps on minibatches drawn on the device by a counter-based
//                      generator (SplitMix64) and gathered by a kernel;
//   sph_relax_run      proposal applications judged by the residual, plain relaxation
//                      to the target, and the pure plain run as the fallback.
// These calls orchestrate libsph's own kernels and entry points from the host; no step of
// the path leaves the GPU.
#include <math.h>

#include <algorithm>

#include "common.cuh"

namespace {

constexpr int kFeat = 128;   // feature width of sph_mlp_features
constexpr int kOut = 3;

// SplitMix64: the generator of Steele, Lea and Flood ("Fast splittable pseudorandom number
// generators", OOPSLA 2014) with the 64-bit mixing function of its public reference
// implementation (Stafford's variant 13): a counter-based stream.
__host__ __device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// targets[i][a] = (x1[a][i] - x0[a][i]) / h, rounded to float32
__global__ void k_delta_over_h(const double* __restrict__ x1, const double* __restrict__ x0, int64_t n, double h,
                               float* __restrict__ out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
#pragma unroll
    for (int a = 0; a < 3; ++a) out[3 * i + a] = (float)((x1[a * n + i] - x0[a * n + i]) / h);
}

// Minibatch of step `step`: row b takes sample splitmix64(key + b) * rows >> 64, with
// key = splitmix64(seed ^ splitmix64(step)).  One warp per row: 128 features as float4.
__global__ void k_gather_batch(const float* __restrict__ feats, const float* __restrict__ targets, int64_t rows,
                               int64_t batch, uint64_t key, float* __restrict__ bf, float* __restrict__ bt) {
    const int64_t b = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (b >= batch) return;
    const uint64_t z = splitmix64(key + (uint64_t)b);
    const int64_t r = (int64_t)__umul64hi(z, (uint64_t)rows);
    reinterpret_cast<float4*>(bf + b * kFeat)[lane] = reinterpret_cast<const float4*>(feats + r * kFeat)[lane];
    if (lane < kOut) bt[b * kOut + lane] = targets[r * kOut + lane];
}

}  // namespace

extern "C" int sph_relax_samples(sph_ctx* ctx, const sph_relax_params* p, double* pos, const double* vol,
                                 int snapshots, int every, float* feats, float* targets, void* stream) {
    if (!ctx || !p || snapshots < 0 || every < 1) return SPH_ERR_ARG;
    const int64_t n = p->dom.n;
    if (n < 0 || p->dom.dim != 3) return SPH_ERR_ARG;
    if (n == 0 || snapshots == 0) return SPH_OK;
    if (!pos || !vol || !feats || !targets) return SPH_ERR_ARG;
    cudaStream_t s = as_stream(stream);
    int st = SPH_OK;
    double* x0 = (double*)sph_scratch(ctx, S_LEARN0, (size_t)n * 3 * 8, &st);
    if (st) return st;
    for (int k = 0; k < snapshots; ++k) {
        st = sph_mlp_features(ctx, p, pos, feats + (size_t)k * n * kFeat, stream);
        if (st) return st;
        SPH_CUDA(ctx, cudaMemcpyAsync(x0, pos, (size_t)n * 3 * 8, cudaMemcpyDeviceToDevice, s));
        st = sph_relax_step(ctx, p, pos, vol, every, stream);
        if (st) return st;
        k_delta_over_h<<<grid_for(n, 256), 256, 0, s>>>(pos, x0, n, p->dom.h, targets + (size_t)k * n * kOut);
        SPH_LAUNCH_CHECK(ctx);
    }
    return SPH_OK;
}

extern "C" int sph_mlp_train(sph_ctx* ctx, float* params, float* adam_m, float* adam_v, int64_t first_step, double lr,
                             const float* feats, const float* targets, int64_t rows, int64_t batch, int nsteps,
                             uint64_t seed, double* loss_host, void* stream) {
    if (!ctx || nsteps < 0 || first_step < 1 || rows < 1 || batch < 1 || batch > (1 << 22)) return SPH_ERR_ARG;
    if (!params || !adam_m || !adam_v || !feats || !targets) return SPH_ERR_ARG;
    if (nsteps == 0) return SPH_OK;
    cudaStream_t s = as_stream(stream);
    int st = SPH_OK;
    float* bf = (float*)sph_scratch(ctx, S_LEARN1, (size_t)batch * (kFeat + kOut) * 4 + 256, &st);
    if (st) return st;
    float* bt = bf + (size_t)batch * kFeat;
    for (int k = 0; k < nsteps; ++k) {
        const uint64_t step = (uint64_t)(first_step + k);
        const uint64_t key = splitmix64(seed ^ splitmix64(step));
        k_gather_batch<<<grid_for(batch * 32, 256), 256, 0, s>>>(feats, targets, rows, batch, key, bf, bt);
        SPH_LAUNCH_CHECK(ctx);
        st = sph_mlp_train_step(ctx, params, adam_m, adam_v, (int64_t)step, lr, bf, bt, batch,
                                k == nsteps - 1 ? loss_host : nullptr, stream);
        if (st) return st;
    }
    return SPH_OK;
}

extern "C" int sph_relax_run(sph_ctx* ctx, const sph_relax_params* p, double* pos, const double* vol,
                             const sph_relax_run_params* rp, sph_relax_run_result* out, void* stream) {
    if (!ctx || !p || !rp || !out) return SPH_ERR_ARG;
    if (rp->max_steps < 0 || rp->check_every < 1 || rp->applications < 0 || rp->plain_between < 0) return SPH_ERR_ARG;
    if (!(rp->target >= 0.0)) return SPH_ERR_ARG;
    if (rp->applications > 0 && (!rp->proposal || p->dom.dim != 3)) return SPH_ERR_ARG;
    const int64_t n = p->dom.n;
    if (n < 0) return SPH_ERR_ARG;
    if (n > 0 && (!pos || !vol)) return SPH_ERR_ARG;
    if (rp->judge != SPH_FP64 && rp->judge != SPH_FP32_KAHAN) return SPH_ERR_ARG;
    cudaStream_t s = as_stream(stream);
    *out = sph_relax_run_result{};
    // the residual that judges: float64 throughout, or from the float32 pair sums
    auto judge = [&](double* r) {
        return rp->judge == SPH_FP64 ? sph_relax_residual(ctx, p, pos, vol, r, stream)
                                     : sph_relax_residual_fp32(ctx, p, pos, vol, r, stream);
    };
    double r3[3] = {0.0, 0.0, 0.0};
    int st = judge(r3);
    if (st) return st;
    const size_t bytes = (size_t)n * p->dom.dim * 8;
    double* start = nullptr;
    double* saved = nullptr;
    if (rp->applications > 0 && n > 0) {
        start = (double*)sph_scratch(ctx, S_LEARN0, bytes + 256, &st);
        if (st) return st;
        saved = (double*)sph_scratch(ctx, S_LEARN2, bytes + 256, &st);
        if (st) return st;
        SPH_CUDA(ctx, cudaMemcpyAsync(start, pos, bytes, cudaMemcpyDeviceToDevice, s));
    }
    // plain steps in chunks of check_every until the target or `budget` steps
    auto plain = [&](int budget) -> int {
        int done = 0;
        while (r3[0] > rp->target && done < budget) {
            const int k = std::min(rp->check_every, budget - done);
            int e = sph_relax_step(ctx, p, pos, vol, k, stream);
            if (e) return e;
            done += k;
            out->steps += k;
            e = judge(r3);
            if (e) return e;
        }
        return SPH_OK;
    };
    bool proposing = rp->applications > 0;
    for (int a = 0; proposing && a < rp->applications && r3[0] > rp->target; ++a) {
        const double before[3] = {r3[0], r3[1], r3[2]};
        SPH_CUDA(ctx, cudaMemcpyAsync(saved, pos, bytes, cudaMemcpyDeviceToDevice, s));
        st = sph_relax_propose(ctx, p, rp->proposal, pos, stream);
        if (st) return st;
        st = sph_take_status(ctx, stream);      // the fused forward's bounded waits
        if (st) return st;
        st = judge(r3);
        if (st) return st;
        if (!(r3[0] < before[0])) {
            // the residual judges the proposal: undo it and go on with plain relaxation
            SPH_CUDA(ctx, cudaMemcpyAsync(pos, saved, bytes, cudaMemcpyDeviceToDevice, s));
            for (int k = 0; k < 3; ++k) r3[k] = before[k];
            out->proposals_rejected += 1;
            proposing = false;
            break;
        }
        out->proposals_kept += 1;
        st = plain(std::min(rp->plain_between, rp->max_steps - out->steps));
        if (st) return st;
    }
    st = plain(rp->max_steps - out->steps);
    if (st) return st;
    if (r3[0] > rp->target && rp->applications > 0 && n > 0) {
        // the learned run missed the target within the cap: plain relaxation from the
        // start is the fallback, and its result is the call's
        SPH_CUDA(ctx, cudaMemcpyAsync(pos, start, bytes, cudaMemcpyDeviceToDevice, s));
        out->fell_back = 1;
        out->steps_before_fallback = out->steps;
        out->steps = 0;
        st = judge(r3);
        if (st) return st;
        st = plain(rp->max_steps);
        if (st) return st;
    }
    out->reached = r3[0] <= rp->target ? 1 : 0;
    out->judged = r3[0];
    // the result's residual in float64 (both kernels)
    st = sph_relax_residual(ctx, p, pos, vol, r3, stream);
    if (st) return st;
    for (int k = 0; k < 3; ++k) out->residual[k] = r3[k];
    return SPH_OK;
}
