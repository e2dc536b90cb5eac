// Context, scratch arena, validation, cell grid, device-wide scan and the
// kernel-evaluation entry point of libsph.
#include <math.h>
#include <new>
#include "common.cuh"
#include <mutex>
#include <set>
#include <utility>

extern "C" int sph_create(sph_ctx** out, int device) {
    if (!out) return SPH_ERR_ARG;
    *out = nullptr;
    sph_ctx* ctx = new (std::nothrow) sph_ctx();
    if (!ctx) return SPH_ERR_ARG;
    ctx->device = device;
    cudaError_t e = cudaSetDevice(device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device);
    if (e == cudaSuccess) e = cudaMalloc((void**)&ctx->flags, FLAG_COUNT * sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(ctx->flags, 0, FLAG_COUNT * sizeof(int));
    if (e == cudaSuccess) e = cudaMallocHost(&ctx->pinned, 4096);
    if (e != cudaSuccess) {
        if (ctx->flags) cudaFree(ctx->flags);
        delete ctx;
        return SPH_ERR_CUDA;
    }
    *out = ctx;
    return SPH_OK;
}

// Gives the persisting L2 set-aside back (and turns the lines marked persisting to normal);
// the caller has synchronised the device, as the reset is not ordered with any stream.
static void l2_release(sph_ctx* ctx) {
    if (!ctx->l2_setaside) return;
    cudaCtxResetPersistingL2Cache();
    cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, 0);
    cudaGetLastError();
    ctx->l2_setaside = 0;
}

L2Win sph_l2_window(sph_ctx* ctx, const void* base, size_t bytes, size_t total) {
    L2Win w;
    if (!ctx->l2_persist || !base || !bytes || !total) return w;
    if (!ctx->l2_setaside) {
        int most = 0, win = 0;
        if (cudaDeviceGetAttribute(&most, cudaDevAttrMaxPersistingL2CacheSize, ctx->device) != cudaSuccess ||
            cudaDeviceGetAttribute(&win, cudaDevAttrMaxAccessPolicyWindowSize, ctx->device) != cudaSuccess ||
            most <= 0 || win <= 0) {
            cudaGetLastError();
            ctx->l2_persist = 0;
            return w;
        }
        const size_t want = total < (size_t)most ? total : (size_t)most;
        size_t got = 0;
        if (cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, want) != cudaSuccess ||
            cudaDeviceGetLimit(&got, cudaLimitPersistingL2CacheSize) != cudaSuccess || got == 0) {
            cudaGetLastError();
            ctx->l2_persist = 0;
            return w;
        }
        ctx->l2_setaside = got;
        ctx->l2_max_window = (size_t)win;
    }
    w.base = base;
    w.bytes = bytes < ctx->l2_max_window ? bytes : ctx->l2_max_window;
    const double hit = (double)ctx->l2_setaside / (double)total;
    w.hit = hit >= 1.0 ? 1.0f : (float)hit;
    return w;
}

extern "C" int sph_set_l2_persist(sph_ctx* ctx, int on) {
    if (!ctx || (on != 0 && on != 1)) return SPH_ERR_ARG;
    if (!on && ctx->l2_setaside) {
        cudaSetDevice(ctx->device);
        if (cudaDeviceSynchronize() != cudaSuccess) {
            cudaGetLastError();
            return SPH_ERR_CUDA;
        }
        l2_release(ctx);
    }
    ctx->l2_persist = on;
    return SPH_OK;
}

extern "C" int sph_destroy(sph_ctx* ctx) {
    if (!ctx) return SPH_ERR_ARG;
    cudaSetDevice(ctx->device);
    cudaDeviceSynchronize();
    l2_release(ctx);
    for (auto& r : ctx->pending) { ctx->pool.push_back(r.start); ctx->pool.push_back(r.stop); }
    ctx->pending.clear();
    for (cudaEvent_t e : ctx->pool) cudaEventDestroy(e);
    ctx->pool.clear();
    if (ctx->batch_graph) cudaGraphExecDestroy(ctx->batch_graph);
    if (ctx->capture_stream) cudaStreamDestroy(ctx->capture_stream);
    if (ctx->side_stream) cudaStreamDestroy(ctx->side_stream);
    for (cudaEvent_t e : ctx->side_ev)
        if (e) cudaEventDestroy(e);
    for (int i = 0; i < sph_ctx::kSlots; ++i)
        if (ctx->slot_ptr[i]) cudaFree(ctx->slot_ptr[i]);
    if (ctx->flags) cudaFree(ctx->flags);
    if (ctx->pinned) cudaFreeHost(ctx->pinned);
    delete ctx;
    return SPH_OK;
}

extern "C" const char* sph_status_string(int status) {
    switch (status) {
        case SPH_OK: return "SPH_OK";
        case SPH_ERR_ARG: return "SPH_ERR_ARG: invalid argument";
        case SPH_ERR_CAPACITY: return "SPH_ERR_CAPACITY: output capacity too small";
        case SPH_ERR_CUDA: return "SPH_ERR_CUDA: CUDA runtime error";
        case SPH_ERR_TIMEOUT: return "SPH_ERR_TIMEOUT: bounded device wait expired";
        case SPH_ERR_NONFINITE: return "SPH_ERR_NONFINITE: non-finite value in a reduction";
        case SPH_ERR_LIMIT: return "SPH_ERR_LIMIT: input exceeds the fixed size of the static scratch array";
        default: return "unknown status";
    }
}

extern "C" int sph_last_cuda_error(const sph_ctx* ctx) { return ctx ? ctx->last_cuda_error : 0; }

extern "C" int sph_set_lanes(sph_ctx* ctx, int pass, int lanes) {
    if (!ctx || pass < 0 || pass > SPH_PASS_COMPRESSIBLE) return SPH_ERR_ARG;
    if (lanes != 1 && lanes != 2 && lanes != 4 && lanes != 8) return SPH_ERR_ARG;
    ctx->lanes[pass] = lanes;
    return SPH_OK;
}

extern "C" int sph_get_lanes(const sph_ctx* ctx, int pass) {
    if (!ctx || pass < 0 || pass > SPH_PASS_COMPRESSIBLE) return -1;
    return ctx->lanes[pass];
}

extern "C" int sph_set_relax_skin(sph_ctx* ctx, double skin_over_h) {
    if (!ctx || !(skin_over_h >= 0.0 && skin_over_h <= 1.0)) return SPH_ERR_ARG;
    ctx->relax_skin = skin_over_h;
    return SPH_OK;
}

extern "C" int sph_set_tile_pipeline(sph_ctx* ctx, int mode) {
    if (!ctx || mode < SPH_PIPE_STREAM || mode > SPH_PIPE_GEOM) return SPH_ERR_ARG;
    ctx->tile_pipe = mode;
    return SPH_OK;
}

extern "C" int sph_set_wait_test(sph_ctx* ctx, uint32_t polls) {
    if (!ctx || polls > (1u << 16)) return SPH_ERR_ARG;
    ctx->wait_test_polls = polls;
    return SPH_OK;
}

// Reads and clears the device timeout flag (synchronises the stream).
int sph_take_timeout(sph_ctx* ctx, cudaStream_t s) {
    int* h = (int*)ctx->pinned;
    SPH_CUDA(ctx, cudaMemcpyAsync(h, ctx->flags + FLAG_TIMEOUT, sizeof(int), cudaMemcpyDeviceToHost, s));
    SPH_CUDA(ctx, cudaStreamSynchronize(s));
    if (*h) {
        SPH_CUDA(ctx, cudaMemsetAsync(ctx->flags + FLAG_TIMEOUT, 0, sizeof(int), s));
        return SPH_ERR_TIMEOUT;
    }
    return SPH_OK;
}

extern "C" int sph_host_alloc(size_t bytes, void** host, void** dev) {
    if (!host || !dev || bytes == 0) return SPH_ERR_ARG;
    *host = nullptr;
    *dev = nullptr;
    void* h = nullptr;
    if (cudaHostAlloc(&h, bytes, cudaHostAllocMapped | cudaHostAllocPortable) != cudaSuccess) {
        cudaGetLastError();
        return SPH_ERR_CUDA;
    }
    void* d = nullptr;
    if (cudaHostGetDevicePointer(&d, h, 0) != cudaSuccess) {
        cudaGetLastError();
        cudaFreeHost(h);
        return SPH_ERR_CUDA;
    }
    *host = h;
    *dev = d;
    return SPH_OK;
}

extern "C" int sph_host_free(void* host) {
    if (!host) return SPH_ERR_ARG;
    return cudaFreeHost(host) == cudaSuccess ? SPH_OK : SPH_ERR_CUDA;
}

extern "C" int sph_set_stage_cap(sph_ctx* ctx, int cap) {
    if (!ctx || cap < 0) return SPH_ERR_ARG;
    ctx->stage_cap = cap;
    return SPH_OK;
}

extern "C" int sph_set_entry_ring(sph_ctx* ctx, int mode) {
    if (!ctx || (mode != SPH_RING_AUTO && mode != SPH_RING_THREAD && mode != SPH_RING_CHUNK)) return SPH_ERR_ARG;
    ctx->entry_ring = mode;
    return SPH_OK;
}

static cudaEvent_t pool_get(sph_ctx* ctx) {
    if (!ctx->pool.empty()) {
        cudaEvent_t e = ctx->pool.back();
        ctx->pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

int sph_timer_begin(sph_ctx* ctx, int slot, cudaStream_t s) {
    if (ctx->timing <= 0) return -1;
    const long long c = ctx->t_all[slot]++;
    if (c % ctx->timing) return -1;                // not a sampled launch
    TimerRec r;
    r.slot = slot;
    r.start = pool_get(ctx);
    r.stop = pool_get(ctx);
    if (!r.start || !r.stop) return -1;
    cudaEventRecord(r.start, s);
    ctx->pending.push_back(r);
    return (int)ctx->pending.size() - 1;
}

void sph_timer_end(sph_ctx* ctx, int token, cudaStream_t s) {
    if (token < 0 || token >= (int)ctx->pending.size()) return;
    cudaEventRecord(ctx->pending[token].stop, s);
}

static int drain_timers(sph_ctx* ctx) {
    for (auto& r : ctx->pending) {
        float ms = 0.0f;
        cudaError_t e = cudaEventSynchronize(r.stop);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, r.start, r.stop);
        if (e != cudaSuccess) { ctx->last_cuda_error = (int)e; ctx->pending.clear(); return SPH_ERR_CUDA; }
        ctx->t_ms[r.slot] += ms;
        ctx->t_n[r.slot] += 1;
        ctx->pool.push_back(r.start);
        ctx->pool.push_back(r.stop);
    }
    ctx->pending.clear();
    return SPH_OK;
}

extern "C" int sph_timing_enable(sph_ctx* ctx, int on) {
    if (!ctx) return SPH_ERR_ARG;
    int st = drain_timers(ctx);
    if (on < 0) return SPH_ERR_ARG;
    for (int k = 0; k < SPH_TIMER_SLOTS; ++k) { ctx->t_ms[k] = 0.0; ctx->t_n[k] = 0; ctx->t_all[k] = 0; }
    ctx->timing = on;
    return st;
}

extern "C" int sph_timing_launches(const sph_ctx* ctx, int slot, int64_t* launches_host) {
    if (!ctx || slot < 0 || slot >= SPH_TIMER_SLOTS || !launches_host) return SPH_ERR_ARG;
    *launches_host = ctx->t_all[slot];
    return SPH_OK;
}

extern "C" int sph_timing_read(sph_ctx* ctx, int slot, double* total_ms_host, int64_t* launches_host) {
    if (!ctx || slot < 0 || slot >= SPH_TIMER_SLOTS || !total_ms_host || !launches_host) return SPH_ERR_ARG;
    int st = drain_timers(ctx);
    *total_ms_host = ctx->t_ms[slot];
    *launches_host = ctx->t_n[slot];
    return st;
}

void* sph_scratch(sph_ctx* ctx, int slot, size_t bytes, int* status) {
    if (bytes == 0) bytes = 16;
    if (ctx->slot_bytes[slot] >= bytes) return ctx->slot_ptr[slot];
    if (ctx->slot_ptr[slot]) {
        cudaError_t e = cudaFree(ctx->slot_ptr[slot]);
        ctx->slot_ptr[slot] = nullptr;
        ctx->slot_bytes[slot] = 0;
        if (e != cudaSuccess) { ctx->last_cuda_error = (int)e; *status = SPH_ERR_CUDA; return nullptr; }
    }
    size_t grow = bytes + bytes / 4 + 256;
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, grow);
    if (e != cudaSuccess) { ctx->last_cuda_error = (int)e; *status = SPH_ERR_CUDA; return nullptr; }
    ctx->slot_ptr[slot] = p;
    ctx->slot_bytes[slot] = grow;
    return p;
}

int sph_check_domain(const sph_domain* dom) {
    if (!dom) return SPH_ERR_ARG;
    if (dom->dim != 2 && dom->dim != 3) return SPH_ERR_ARG;
    if (dom->n < 0 || dom->n > 0x7fffffffLL) return SPH_ERR_ARG;
    if (!(dom->h > 0.0) || !isfinite(dom->h)) return SPH_ERR_ARG;
    if (!(dom->kappa > 0.0) || !(dom->kappa <= 2.0)) return SPH_ERR_ARG;
    double rc = dom->kappa * dom->h;
    for (int k = 0; k < dom->dim; ++k) {
        if (!(dom->len[k] > 0.0) || !isfinite(dom->len[k]) || !isfinite(dom->lo[k])) return SPH_ERR_ARG;
        if (((dom->periodic_mask >> k) & 1u) && dom->len[k] < 2.0 * rc) return SPH_ERR_ARG;
    }
    if (dom->periodic_mask >> dom->dim) return SPH_ERR_ARG;
    return SPH_OK;
}

CellGrid sph_make_grid(const sph_domain* dom) {
    CellGrid g;
    g.dim = dom->dim;
    double rc = dom->kappa * dom->h;
    g.rc2 = rc * rc;
    g.total = 1;
    g.periodic = dom->periodic_mask;
    for (int k = 0; k < 3; ++k) {
        if (k < dom->dim) {
            double m = floor(dom->len[k] / rc);
            if (m < 1.0) m = 1.0;
            if (m > 1048576.0) m = 1048576.0;
            g.n[k] = (int)m;
            g.size[k] = dom->len[k] / (double)g.n[k];
            g.lo[k] = dom->lo[k];
            g.len[k] = dom->len[k];
            g.half[k] = 0.5 * dom->len[k];
        } else {
            g.n[k] = 1; g.size[k] = 1.0; g.lo[k] = 0.0; g.len[k] = 1.0; g.half[k] = 0.5;
        }
        g.total *= g.n[k];
    }
    return g;
}

// ---------------------------------------------------------------------------
// Device-wide exclusive scan: per-block sums, a single-block scan of the block
// sums, then a per-block rescan with the block offset.
static const int SCAN_THREADS = 256;
static const int SCAN_ITEMS = 8;
static const int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

template <typename T>
__device__ T block_exclusive_scan(T v, T* total) {
    __shared__ T warp_sums[32];
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[warp] = x;
    __syncthreads();
    int nw = blockDim.x >> 5;
    if (warp == 0) {
        T w = lane < nw ? warp_sums[lane] : T(0);
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            T y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < nw) warp_sums[lane] = w;
    }
    __syncthreads();
    T before = warp > 0 ? warp_sums[warp - 1] : T(0);
    *total = warp_sums[nw - 1];
    __syncthreads();
    return before + x - v;
}

template <typename T>
__global__ void k_scan_block_sums(const int32_t* in, int64_t n, T* bsum) {
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
    T s = 0;
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        int64_t idx = base + (int64_t)threadIdx.x * SCAN_ITEMS + k;
        if (idx < n) s += (T)in[idx];
    }
    T tot;
    block_exclusive_scan<T>(s, &tot);
    if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

template <typename T>
__global__ void k_scan_bsums(T* bsum, int64_t nb) {
    T carry = 0;
    for (int64_t base = 0; base < nb; base += blockDim.x) {
        int64_t idx = base + threadIdx.x;
        T v = idx < nb ? bsum[idx] : T(0);
        T tot;
        T ex = block_exclusive_scan<T>(v, &tot);
        if (idx < nb) bsum[idx] = ex + carry;
        carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) bsum[nb] = carry;
}

template <typename T>
__global__ void k_scan_apply(const int32_t* in, int64_t n, const T* bsum, T* out) {
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
    T vals[SCAN_ITEMS];
    T s = 0;
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        int64_t idx = base + k;
        vals[k] = idx < n ? (T)in[idx] : T(0);
        s += vals[k];
    }
    T tot;
    T ex = block_exclusive_scan<T>(s, &tot) + bsum[blockIdx.x];
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        int64_t idx = base + k;
        if (idx < n) out[idx] = ex;
        ex += vals[k];
    }
}

template <typename T>
__global__ void k_scan_total(const T* bsum, int64_t nb, T* out, int64_t n) { out[n] = bsum[nb]; }

template <typename T>
static int scan_impl(sph_ctx* ctx, const int32_t* in, T* out, int64_t n, cudaStream_t s) {
    int64_t nb = (n + SCAN_TILE - 1) / SCAN_TILE;
    if (nb < 1) nb = 1;
    int st = SPH_OK;
    T* bsum = (T*)sph_scratch(ctx, S_SCAN_BLOCKS, (size_t)(nb + 1) * sizeof(T), &st);
    if (!bsum) return st;
    k_scan_block_sums<T><<<(unsigned)nb, SCAN_THREADS, 0, s>>>(in, n, bsum);
    k_scan_bsums<T><<<1, 1024, 0, s>>>(bsum, nb);
    k_scan_apply<T><<<(unsigned)nb, SCAN_THREADS, 0, s>>>(in, n, bsum, out);
    k_scan_total<T><<<1, 1, 0, s>>>(bsum, nb, out, n);
    SPH_LAUNCH_CHECK(ctx);
    return SPH_OK;
}

// Same scan with a caller-provided block-sum buffer of at least
// (n / 2048 + 2) elements (used by the allocation-free neighbour build).
template <typename T>
static int scan_with_buffer(const int32_t* in, T* out, int64_t n, T* bsum, cudaStream_t s) {
    int64_t nb = (n + SCAN_TILE - 1) / SCAN_TILE;
    if (nb < 1) nb = 1;
    k_scan_block_sums<T><<<(unsigned)nb, SCAN_THREADS, 0, s>>>(in, n, bsum);
    k_scan_bsums<T><<<1, 1024, 0, s>>>(bsum, nb);
    k_scan_apply<T><<<(unsigned)nb, SCAN_THREADS, 0, s>>>(in, n, bsum, out);
    k_scan_total<T><<<1, 1, 0, s>>>(bsum, nb, out, n);
    return cudaGetLastError() == cudaSuccess ? SPH_OK : SPH_ERR_CUDA;
}

int sph_exclusive_scan_i64_buf(const int32_t* in, int64_t* out, int64_t n, int64_t* bsum, cudaStream_t s) {
    return scan_with_buffer<long long>(in, (long long*)out, n, (long long*)bsum, s);
}
int sph_exclusive_scan_i32_buf(const int32_t* in, int32_t* out, int64_t n, int32_t* bsum, cudaStream_t s) {
    return scan_with_buffer<int>(in, (int*)out, n, (int*)bsum, s);
}

int sph_exclusive_scan_i64(sph_ctx* ctx, const int32_t* in, int64_t* out, int64_t n, cudaStream_t s) {
    return scan_impl<long long>(ctx, in, (long long*)out, n, s);
}
int sph_exclusive_scan_i32(sph_ctx* ctx, const int32_t* in, int32_t* out, int64_t n, cudaStream_t s) {
    return scan_impl<int>(ctx, in, (int*)out, n, s);
}

// ---------------------------------------------------------------------------
// a3: kernel values and derivatives (Eqs. 6 and 8).
template <typename R>
__global__ void k_kernel_eval(int kernel, int dim, R h, R kappa, R alpha, const double* r,
                              double* w, double* dwdr, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    R q = (R)r[i] / h;
    R hd = dim == 2 ? h * h : h * h * h;
    R wv = R(0), dv = R(0);
    if (q <= kappa) {
        if (kernel == SPH_WENDLAND_C2) {
            R t = R(1) - R(0.5) * q;
            R t3 = t * t * t;
            wv = alpha / hd * (t3 * t) * (R(2) * q + R(1));
            dv = alpha / (hd * h) * (R(-5) * q) * t3;
        } else {
            R q2 = q * q;
            R e = exp(-q2);
            wv = alpha / hd * (R(1) - R(0.5) * q2 + q2 * q2 / R(6)) * e;
            dv = -alpha / (hd * h) * (q / R(3)) * e * (R(9) - R(5) * q2 + q2 * q2);
        }
    }
    if (w) w[i] = (double)wv;
    if (dwdr) dwdr[i] = (double)dv;
}

extern "C" int sph_kernel_eval(int kernel, int dim, double h, double kappa, int precision,
                               const double* r, double* w, double* dwdr, int64_t n, void* stream) {
    if (kernel != SPH_WENDLAND_C2 && kernel != SPH_LAGUERRE_GAUSS) return SPH_ERR_ARG;
    if (dim != 2 && dim != 3) return SPH_ERR_ARG;
    if (!(h > 0.0) || !(kappa > 0.0) || kappa > 2.0 || n < 0) return SPH_ERR_ARG;
    if (precision != SPH_FP64 && precision != SPH_FP32_KAHAN) return SPH_ERR_ARG;
    if (n == 0) return SPH_OK;
    if (!r) return SPH_ERR_ARG;
    double alpha = kernel == SPH_WENDLAND_C2 ? wendland_alpha(dim) : lg_alpha(dim);
    cudaStream_t s = as_stream(stream);
    if (precision == SPH_FP64)
        k_kernel_eval<double><<<grid_for(n, 256), 256, 0, s>>>(kernel, dim, h, kappa, alpha, r, w, dwdr, n);
    else
        k_kernel_eval<float><<<grid_for(n, 256), 256, 0, s>>>(kernel, dim, (float)h, (float)kappa,
                                                              (float)alpha, r, w, dwdr, n);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? SPH_OK : SPH_ERR_CUDA;
}

void sph_allow_dynamic_smem(const void* kernel) {
    static std::mutex mu;
    static std::set<std::pair<const void*, int>> done;
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lock(mu);
    if (done.insert({kernel, dev}).second)
        cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
}

extern "C" int sph_take_status(sph_ctx* ctx, void* stream) {
    if (!ctx) return SPH_ERR_ARG;
    ctx->waits_pending = false;
    return sph_take_timeout(ctx, as_stream(stream));
}
