// a13: many independent Eulerian cases of uneven size advanced together.
//
// All cases' packed float32 records and CSR lists are concatenated.  One
// persistent launch per pass (momentum, then continuity) walks the
// concatenated particle range in fixed-size tiles (tile t -> block t mod grid,
// a static schedule, so results are deterministic and match the single-case
// kernel's to float32 rounding).  Each group of LANES lanes finds its particle's case by
// binary search over the case offsets kept in shared memory together with the
// per-case constants (h, dt, viscosity, box).  The two launches of a step are
// captured once into a CUDA graph and replayed per step.  An autotuner times
// the launch shapes (lanes per particle x block size) on the caller's data and
// keeps the fastest in the context.
#include <cstring>
#include <vector>
#include "common.cuh"
#include "euler_core.cuh"
#include "tiles.cuh"

using namespace euler;

namespace {

constexpr int kMaxCases = 256;

template <int DIM, int MODE, int OUT, int LANES>
__global__ void __launch_bounds__(256) k_euler32_batched(const float* __restrict__ Rin, float* __restrict__ Rout,
                                                         const int64_t* __restrict__ row_ptr,
                                                         const int32_t* __restrict__ col, int64_t ntotal, int ncases,
                                                         const EulerK<float>* __restrict__ cases,
                                                         const int64_t* __restrict__ offsets) {
    __shared__ EulerK<float> sK[kMaxCases];
    __shared__ int64_t sOff[kMaxCases + 1];
    for (int c = threadIdx.x; c < ncases; c += blockDim.x) sK[c] = cases[c];
    for (int c = threadIdx.x; c <= ncases; c += blockDim.x) sOff[c] = offsets[c];
    __syncthreads();
    constexpr int NS = NSym<DIM>::v;
    const int per_block = blockDim.x / LANES;
    const int lane = threadIdx.x % LANES;
    for (int64_t base = (int64_t)blockIdx.x * per_block; base < ntotal; base += (int64_t)gridDim.x * per_block) {
        int64_t i = base + threadIdx.x / LANES;
        bool active = i < ntotal;
        int64_t ii = active ? i : 0;
        // case of particle ii: largest c with sOff[c] <= ii
        int lo = 0, hi = ncases - 1;
        while (lo < hi) {
            int mid = (lo + hi + 1) >> 1;
            if (sOff[mid] <= ii) lo = mid;
            else hi = mid - 1;
        }
        const EulerK<float>& K = sK[lo];
        F8 ma = ldg8(Rin + kRecWords * ii), mb = ldg8(Rin + kRecWords * ii + 8);
        float oi[DIM], Vi, Bi[NS], vi[DIM], dri;
        uint32_t bi;
        unpack_rec<DIM>(ma, mb, oi, bi, Vi, Bi, vi, dri);
        int64_t b = active ? row_ptr[ii] : 0, e = active ? row_ptr[ii + 1] : 0;
        float rm, rp[DIM];
        euler_row32<DIM, MODE, LANES, true>(Rin, col, b, e, lane, oi, bi, Bi, vi, dri, K, rm, rp);
        if (active && lane == 0) {
            float vn[DIM], drn;
            euler_update32<DIM, OUT>(vi, dri, rm, rp, K, vn, drn);
            store_dyn<DIM>(Rout, i, vn, drn);
        }
    }
}

// Planned form (every case carries a tile plan of its own lists, see
// sph_eulerian_plan): one block per tile of any case, the tiles of case c being
// blocks tile0[c] .. tile0[c] + ceil(n_c / kTileRows) - 1 of the launch.
struct PlanCase {
    GeoArgsE A;
    int64_t offset, n, tile0;
};

template <int DIM, int MODE, int OUT, bool CHUNK>
__global__ void __launch_bounds__(kTileRows, 6) k_euler32g_batched(const float* __restrict__ Rin,
                                                                   float* __restrict__ Rout,
                                                                   const int64_t* __restrict__ row_ptr, int ncases,
                                                                   const EulerK<float>* __restrict__ cases,
                                                                   const PlanCase* __restrict__ plans,
                                                                   int* __restrict__ flags) {
    extern __shared__ __align__(16) unsigned char eb_smem[];
    // momentum pass in reverse tile order, continuity pass forwards (pair entries reused from L2)
    const int64_t b = MODE == WANT_MOM ? gridDim.x - 1 - blockIdx.x : blockIdx.x;
    int lo = 0, hi = ncases - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (plans[mid].tile0 <= b) lo = mid;
        else hi = mid - 1;
    }
    const PlanCase C = plans[lo];
    const EulerK<float> K = cases[lo];
    euler_tile_g<DIM, MODE, OUT, CHUNK>(Rin, Rout, row_ptr, C.offset, row_ptr[C.offset], C.n, b - C.tile0, K, C.A,
                                        reinterpret_cast<float4*>(eb_smem), nullptr, nullptr, flags);
}

// Launch shape of the planned form: the tile count and a stage capacity common to
// all cases (0 tiles: some case has no plan).
struct PlanShape {
    int64_t tiles;
    int mcap;
    bool chunk;    // the entries through the TMA chunk ring (one launch covers every case's tiles)
};

PlanShape plan_shape(const sph_ctx* ctx, const sph_batch_case* cases, int ncases) {
    PlanShape sh{0, 1, false};
    int32_t maxm = 0;
    for (int c = 0; c < ncases; ++c) {
        if (!cases[c].plan || cases[c].plan_nnz < 1 || cases[c].plan_maxm < 1) return PlanShape{0, 1, false};
        maxm = cases[c].plan_maxm > maxm ? cases[c].plan_maxm : maxm;
        sh.tiles += (cases[c].n + kTileRows - 1) / kTileRows;
    }
    sh.mcap = stage_mcap(maxm, 1, ctx->stage_cap);
    const int64_t waves = kChunkRingWaves * (int64_t)6 * (ctx->num_sms > 0 ? ctx->num_sms : 1);
    sh.chunk = ctx->entry_ring == SPH_RING_CHUNK || (ctx->entry_ring == SPH_RING_AUTO && sh.tiles >= waves);
    return sh;
}

EulerK<float> case_consts(const sph_batch_case& c, int dim) {
    EulerK<float> K;
    double h = c.h;
    double hd2 = dim == 2 ? h * h * h * h : h * h * h * h * h;
    K.coef = (float)(-5.0 * wendland_alpha(dim) / hd2);
    K.inv_h = (float)(1.0 / h);
    K.rho0 = (float)c.rho0;
    K.c0 = (float)c.c0;
    K.inv_c0 = (float)(1.0 / c.c0);
    K.c0sq = (float)(c.c0 * c.c0);
    K.eta = (float)c.eta;
    K.mu2 = (float)(2.0 * c.mu);
    K.eps_h2 = (float)(0.01 * h * h);
    K.dt = (float)c.dt;
    K.periodic = c.periodic_mask;
    sph_domain d = {};
    d.dim = dim;
    d.h = c.h;
    d.periodic_mask = c.periodic_mask;
    for (int a = 0; a < 3; ++a) d.len[a] = c.len[a];
    RelGrid g = make_rel_grid(d);
    for (int a = 0; a < 3; ++a) {
        K.half[a] = (float)(0.5 * c.len[a]);
        K.Lh[a] = (float)c.len[a];
        K.Ll[a] = (float)(c.len[a] - (double)K.Lh[a]);
        K.S[a] = (float)g.S[a];
        K.Sl[a] = (float)(g.S[a] - (double)K.S[a]);
        K.ncell[a] = g.n[a];
    }
    return K;
}

struct BatchPlan {
    int lanes, block, grid;
};

template <int LANES>
void launch_pass(int out, int dim, const BatchPlan& pl, const sph_batch_state* st, int64_t ntotal, int ncases,
                 const EulerK<float>* dK, const int64_t* dOff, const float* rin, float* rout, cudaStream_t s) {
    if (dim == 2) {
        if (out == OUT_MOM)
            k_euler32_batched<2, WANT_MOM, OUT_MOM, LANES><<<pl.grid, pl.block, 0, s>>>(rin, rout, st->row_ptr, st->col,
                                                                                      ntotal, ncases, dK, dOff);
        else
            k_euler32_batched<2, WANT_MASS, OUT_MASS, LANES><<<pl.grid, pl.block, 0, s>>>(rin, rout, st->row_ptr,
                                                                                        st->col, ntotal, ncases, dK, dOff);
    } else {
        if (out == OUT_MOM)
            k_euler32_batched<3, WANT_MOM, OUT_MOM, LANES><<<pl.grid, pl.block, 0, s>>>(rin, rout, st->row_ptr, st->col,
                                                                                      ntotal, ncases, dK, dOff);
        else
            k_euler32_batched<3, WANT_MASS, OUT_MASS, LANES><<<pl.grid, pl.block, 0, s>>>(rin, rout, st->row_ptr,
                                                                                        st->col, ntotal, ncases, dK, dOff);
    }
}

void launch_step(const BatchPlan& pl, int dim, const sph_batch_state* st, int64_t ntotal, int ncases,
                 const EulerK<float>* dK, const int64_t* dOff, cudaStream_t s) {
    float* r0 = st->rec;
    float* r1 = st->rec_tmp;
    switch (pl.lanes) {
        case 1: launch_pass<1>(OUT_MOM, dim, pl, st, ntotal, ncases, dK, dOff, r0, r1, s);
                launch_pass<1>(OUT_MASS, dim, pl, st, ntotal, ncases, dK, dOff, r1, r0, s); break;
        case 2: launch_pass<2>(OUT_MOM, dim, pl, st, ntotal, ncases, dK, dOff, r0, r1, s);
                launch_pass<2>(OUT_MASS, dim, pl, st, ntotal, ncases, dK, dOff, r1, r0, s); break;
        case 8: launch_pass<8>(OUT_MOM, dim, pl, st, ntotal, ncases, dK, dOff, r0, r1, s);
                launch_pass<8>(OUT_MASS, dim, pl, st, ntotal, ncases, dK, dOff, r1, r0, s); break;
        default: launch_pass<4>(OUT_MOM, dim, pl, st, ntotal, ncases, dK, dOff, r0, r1, s);
                 launch_pass<4>(OUT_MASS, dim, pl, st, ntotal, ncases, dK, dOff, r1, r0, s); break;
    }
}

void launch_step_planned(int dim, const sph_batch_state* st, int ncases, const EulerK<float>* dK,
                         const PlanCase* dP, const PlanShape& sh, int* flags, cudaStream_t s) {
    dim3 g((unsigned)sh.tiles), b(kTileRows);
    size_t smem = (size_t)sh.mcap * 16 + kEntryRingBytes;
    float* r0 = st->rec;
    float* r1 = st->rec_tmp;
    if (dim == 2) {
        auto* fm = sh.chunk ? k_euler32g_batched<2, WANT_MOM, OUT_MOM, true> : k_euler32g_batched<2, WANT_MOM, OUT_MOM, false>;
        auto* fc = sh.chunk ? k_euler32g_batched<2, WANT_MASS, OUT_MASS, true>
                            : k_euler32g_batched<2, WANT_MASS, OUT_MASS, false>;
        sph_allow_dynamic_smem((const void*)fm);
        sph_allow_dynamic_smem((const void*)fc);
        fm<<<g, b, smem, s>>>(r0, r1, st->row_ptr, ncases, dK, dP, flags);
        fc<<<g, b, smem, s>>>(r1, r0, st->row_ptr, ncases, dK, dP, flags);
    } else {
        auto* fm = sh.chunk ? k_euler32g_batched<3, WANT_MOM, OUT_MOM, true> : k_euler32g_batched<3, WANT_MOM, OUT_MOM, false>;
        auto* fc = sh.chunk ? k_euler32g_batched<3, WANT_MASS, OUT_MASS, true>
                            : k_euler32g_batched<3, WANT_MASS, OUT_MASS, false>;
        sph_allow_dynamic_smem((const void*)fm);
        sph_allow_dynamic_smem((const void*)fc);
        fm<<<g, b, smem, s>>>(r0, r1, st->row_ptr, ncases, dK, dP, flags);
        fc<<<g, b, smem, s>>>(r1, r0, st->row_ptr, ncases, dK, dP, flags);
    }
}

int check_batch(const sph_batch_case* cases, int ncases, const sph_batch_state* st, int64_t* ntotal, int* dim) {
    if (!cases || !st || ncases < 1 || ncases > kMaxCases) return SPH_ERR_ARG;
    if (!st->row_ptr || !st->col || !st->rec || !st->rec_tmp) return SPH_ERR_ARG;
    if (((uintptr_t)st->rec & 31u) || ((uintptr_t)st->rec_tmp & 31u)) return SPH_ERR_ARG;
    int64_t off = 0;
    *dim = cases[0].dim;
    for (int c = 0; c < ncases; ++c) {
        const sph_batch_case& k = cases[c];
        if (k.dim != *dim || (k.dim != 2 && k.dim != 3)) return SPH_ERR_ARG;
        if (k.offset != off || k.n < 1) return SPH_ERR_ARG;
        if (!(k.h > 0.0) || !(k.dt > 0.0) || !(k.c0 > 0.0) || !(k.rho0 > 0.0) || !(k.mu >= 0.0)) return SPH_ERR_ARG;
        sph_domain d = {};
        d.dim = k.dim;
        d.h = k.h;
        d.periodic_mask = k.periodic_mask;
        for (int a = 0; a < 3; ++a) {
            if (a < k.dim && !(k.len[a] > 0.0)) return SPH_ERR_ARG;
            d.len[a] = k.len[a];
        }
        if (k.periodic_mask >> k.dim) return SPH_ERR_ARG;
        // lists may hold pairs up to the widest support, 2h
        if (!rel_grid_periodic_ok(make_rel_grid(d), k.dim, 2.0 * k.h)) return SPH_ERR_ARG;
        off += k.n;
    }
    *ntotal = off;
    return SPH_OK;
}

// Device copies of the case table and offsets (uploaded when they change).
int upload_cases(sph_ctx* ctx, const sph_batch_case* cases, int ncases, int dim, EulerK<float>** dK, int64_t** dOff,
                 PlanCase** dP, cudaStream_t s, bool* changed) {
    std::vector<EulerK<float>> K(ncases);
    std::vector<int64_t> off(ncases + 1);
    for (int c = 0; c < ncases; ++c) {
        K[c] = case_consts(cases[c], dim);
        off[c] = cases[c].offset;
    }
    off[ncases] = cases[ncases - 1].offset + cases[ncases - 1].n;
    PlanShape sh = plan_shape(ctx, cases, ncases);
    std::vector<PlanCase> P(sh.tiles ? ncases : 0);
    const int chunk_ring = sh.chunk ? 1 : 0;
    int64_t t0 = 0;
    for (size_t c = 0; c < P.size(); ++c) {
        TilePlan tp = tile_plan_view(const_cast<void*>(cases[c].plan), cases[c].n, cases[c].plan_nnz);
        P[c].A = GeoArgsE{tp.tile_m, tp.tile_so, tp.uidx, reinterpret_cast<const float*>(tp.geo), sh.mcap,
                          ctx->wait_test_polls, chunk_ring};
        P[c].offset = cases[c].offset;
        P[c].n = cases[c].n;
        P[c].tile0 = t0;
        t0 += (cases[c].n + kTileRows - 1) / kTileRows;
    }
    // the offsets follow the constants at a 16-byte boundary (int64 loads need 8-byte alignment
    // and sizeof(EulerK<float>) is not a multiple of 8)
    size_t kb = (sizeof(EulerK<float>) * ncases + 15) & ~size_t(15);
    size_t ob = (sizeof(int64_t) * (ncases + 1) + 15) & ~size_t(15), pb = sizeof(PlanCase) * P.size();
    std::vector<unsigned char> blob(kb + ob + pb, 0);
    std::memcpy(blob.data(), K.data(), sizeof(EulerK<float>) * ncases);
    std::memcpy(blob.data() + kb, off.data(), sizeof(int64_t) * (ncases + 1));
    if (pb) std::memcpy(blob.data() + kb + ob, P.data(), pb);
    *changed = blob != ctx->batch_blob;
    int st = SPH_OK;
    unsigned char* d = (unsigned char*)sph_scratch(ctx, S_BATCH, blob.size() + 256, &st);
    if (st) return st;
    if (*changed) {
        // the upload is synchronous with respect to the host buffer (blob is a local)
        SPH_CUDA(ctx, cudaMemcpyAsync(d, blob.data(), blob.size(), cudaMemcpyHostToDevice, s));
        SPH_CUDA(ctx, cudaStreamSynchronize(s));
        ctx->batch_blob = blob;
    }
    *dK = reinterpret_cast<EulerK<float>*>(d);
    *dOff = reinterpret_cast<int64_t*>(d + kb);
    *dP = pb ? reinterpret_cast<PlanCase*>(d + kb + ob) : nullptr;
    return SPH_OK;
}

int blocks_per_sm(int lanes, int block, int dim) {
    int nb = 0;
    cudaError_t e;
    const void* fn;
    if (dim == 2) {
        switch (lanes) {
            case 1: fn = (const void*)k_euler32_batched<2, WANT_MOM, OUT_MOM, 1>; break;
            case 2: fn = (const void*)k_euler32_batched<2, WANT_MOM, OUT_MOM, 2>; break;
            case 8: fn = (const void*)k_euler32_batched<2, WANT_MOM, OUT_MOM, 8>; break;
            default: fn = (const void*)k_euler32_batched<2, WANT_MOM, OUT_MOM, 4>; break;
        }
    } else {
        switch (lanes) {
            case 1: fn = (const void*)k_euler32_batched<3, WANT_MOM, OUT_MOM, 1>; break;
            case 2: fn = (const void*)k_euler32_batched<3, WANT_MOM, OUT_MOM, 2>; break;
            case 8: fn = (const void*)k_euler32_batched<3, WANT_MOM, OUT_MOM, 8>; break;
            default: fn = (const void*)k_euler32_batched<3, WANT_MOM, OUT_MOM, 4>; break;
        }
    }
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, block, 0);
    if (e != cudaSuccess || nb < 1) nb = 1;
    return nb;
}

BatchPlan make_plan(sph_ctx* ctx, int lanes, int block, int dim, int64_t ntotal) {
    BatchPlan pl;
    pl.lanes = lanes;
    pl.block = block;
    int64_t tiles = (ntotal + block / lanes - 1) / (block / lanes);
    int64_t persistent = (int64_t)ctx->num_sms * blocks_per_sm(lanes, block, dim);
    pl.grid = (int)(tiles < persistent ? tiles : persistent);
    if (pl.grid < 1) pl.grid = 1;
    return pl;
}

int run_steps(sph_ctx* ctx, const BatchPlan& pl, int dim, const sph_batch_state* st, int64_t ntotal, int ncases,
              const EulerK<float>* dK, const int64_t* dOff, const PlanCase* dP, const PlanShape& sh, int nsteps,
              bool tables_changed, cudaStream_t s) {
    // (re)capture one step as a graph when anything it depends on changed
    BatchGraphKey key;
    std::memset(&key, 0, sizeof(key));
    key.row_ptr = st->row_ptr; key.col = st->col; key.rec = st->rec; key.rec_tmp = st->rec_tmp;
    key.ntotal = ntotal; key.ncases = ncases; key.lanes = pl.lanes; key.block = pl.block; key.grid = pl.grid;
    key.dK = dK; key.dim = dim;
    if (dP) { key.lanes = sh.chunk ? -1 : 0; key.block = kTileRows; key.grid = sh.mcap; }
    if (!ctx->batch_graph || tables_changed || std::memcmp(&key, &ctx->batch_key, sizeof(key)) != 0) {
        if (ctx->batch_graph) { cudaGraphExecDestroy(ctx->batch_graph); ctx->batch_graph = nullptr; }
        if (!ctx->capture_stream) SPH_CUDA(ctx, cudaStreamCreateWithFlags(&ctx->capture_stream, cudaStreamNonBlocking));
        cudaGraph_t g = nullptr;
        SPH_CUDA(ctx, cudaStreamBeginCapture(ctx->capture_stream, cudaStreamCaptureModeThreadLocal));
        if (dP) launch_step_planned(dim, st, ncases, dK, dP, sh, ctx->flags, ctx->capture_stream);
        else launch_step(pl, dim, st, ntotal, ncases, dK, dOff, ctx->capture_stream);
        cudaError_t e = cudaStreamEndCapture(ctx->capture_stream, &g);
        if (e != cudaSuccess) { ctx->last_cuda_error = (int)e; return SPH_ERR_CUDA; }
        e = cudaGraphInstantiate(&ctx->batch_graph, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) { ctx->batch_graph = nullptr; ctx->last_cuda_error = (int)e; return SPH_ERR_CUDA; }
        ctx->batch_key = key;
    }
    if (dP && sh.chunk) ctx->waits_pending = true;      // the chunk ring's bounded waits
    for (int k = 0; k < nsteps; ++k) {
        int t = sph_timer_begin(ctx, SPH_TIMER_BATCH_STEP, s);
        SPH_CUDA(ctx, cudaGraphLaunch(ctx->batch_graph, s));
        sph_timer_end(ctx, t, s);
    }
    return SPH_OK;
}

}  // namespace

extern "C" int sph_eulerian_step_batched(sph_ctx* ctx, const sph_batch_case* cases, int ncases,
                                         const sph_batch_state* st, int nsteps, void* stream) {
    if (!ctx || nsteps < 0) return SPH_ERR_ARG;
    int64_t ntotal = 0;
    int dim = 0;
    int r = check_batch(cases, ncases, st, &ntotal, &dim);
    if (r) return r;
    if (nsteps == 0) return SPH_OK;
    cudaStream_t s = as_stream(stream);
    EulerK<float>* dK = nullptr;
    int64_t* dOff = nullptr;
    PlanCase* dP = nullptr;
    bool changed = false;
    r = upload_cases(ctx, cases, ncases, dim, &dK, &dOff, &dP, s, &changed);
    if (r) return r;
    PlanShape sh = plan_shape(ctx, cases, ncases);
    BatchPlan pl = make_plan(ctx, ctx->lanes[SPH_PASS_BATCHED], ctx->batch_block, dim, ntotal);
    return run_steps(ctx, pl, dim, st, ntotal, ncases, dK, dOff, dP, sh, nsteps, changed, s);
}

extern "C" int sph_autotune_batched(sph_ctx* ctx, const sph_batch_case* cases, int ncases, const sph_batch_state* st,
                                    int trial_steps, int* lanes_host, int* block_host, double* ms_host,
                                    void* stream) {
    if (!ctx || trial_steps < 1) return SPH_ERR_ARG;
    int64_t ntotal = 0;
    int dim = 0;
    int r = check_batch(cases, ncases, st, &ntotal, &dim);
    if (r) return r;
    cudaStream_t s = as_stream(stream);
    EulerK<float>* dK = nullptr;
    int64_t* dOff = nullptr;
    PlanCase* dP = nullptr;
    bool changed = false;
    r = upload_cases(ctx, cases, ncases, dim, &dK, &dOff, &dP, s, &changed);
    if (r) return r;
    PlanShape sh = plan_shape(ctx, cases, ncases);
    // the trial steps advance the caller's state: it is saved first and restored after every variant
    int64_t qbytes = ntotal * kRecWords * 4;
    void* save = sph_scratch(ctx, S_MISC3, (size_t)qbytes, &r);
    if (r) return r;
    SPH_CUDA(ctx, cudaMemcpyAsync(save, st->rec, qbytes, cudaMemcpyDeviceToDevice, s));
    cudaEvent_t e0, e1;
    SPH_CUDA(ctx, cudaEventCreate(&e0));
    SPH_CUDA(ctx, cudaEventCreate(&e1));
    const int lanes_set[4] = {1, 2, 4, 8};
    const int block_set[2] = {128, 256};
    double best = 1e300;
    int bl = 4, bb = 256;
    for (int li = 0; li < 4; ++li)
        for (int bi = 0; bi < 2; ++bi) {
            BatchPlan pl = make_plan(ctx, lanes_set[li], block_set[bi], dim, ntotal);
            r = run_steps(ctx, pl, dim, st, ntotal, ncases, dK, dOff, dP, sh, 1, changed, s);   // warm + capture
            if (r) return r;
            changed = false;
            SPH_CUDA(ctx, cudaEventRecord(e0, s));
            r = run_steps(ctx, pl, dim, st, ntotal, ncases, dK, dOff, dP, sh, trial_steps, false, s);
            if (r) return r;
            SPH_CUDA(ctx, cudaEventRecord(e1, s));
            SPH_CUDA(ctx, cudaEventSynchronize(e1));
            float ms = 0.0f;
            SPH_CUDA(ctx, cudaEventElapsedTime(&ms, e0, e1));
            if (ms < best) { best = ms; bl = lanes_set[li]; bb = block_set[bi]; }
            SPH_CUDA(ctx, cudaMemcpyAsync(st->rec, save, qbytes, cudaMemcpyDeviceToDevice, s));
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    ctx->lanes[SPH_PASS_BATCHED] = bl;
    ctx->batch_block = bb;
    if (lanes_host) *lanes_host = bl;
    if (block_host) *block_host = bb;
    if (ms_host) *ms_host = best / trial_steps;
    SPH_CUDA(ctx, cudaStreamSynchronize(s));
    return SPH_OK;
}
