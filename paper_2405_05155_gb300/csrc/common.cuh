// Shared device helpers of libsph: context, error plumbing, kernel functions,
// minimum image, compensated sums and a device-wide exclusive scan.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <math.h>
#include <vector>

#include "sph.h"

struct TimerRec {
    int slot;
    cudaEvent_t start, stop;
};

// What a captured batched step depends on (compared bytewise; zero-initialise).
struct BatchGraphKey {
    const void* row_ptr;
    const void* col;
    const void* rec;
    const void* rec_tmp;
    const void* dK;
    int64_t ntotal;
    int ncases, lanes, block, grid, dim, pad;
};

struct sph_ctx {
    // per-kernel timing (sph_timing_enable): events recorded around launches
    int timing = 0;                 // 0: off; k >= 1: every k-th launch of a slot is timed
    std::vector<TimerRec> pending;
    std::vector<cudaEvent_t> pool;
    double t_ms[SPH_TIMER_SLOTS] = {};
    long long t_n[SPH_TIMER_SLOTS] = {};
    long long t_all[SPH_TIMER_SLOTS] = {};   // launches seen while timing was on (timed or not)
    int device = 0;
    int last_cuda_error = 0;
    int num_sms = 0;
    static const int kSlots = 32;
    void* slot_ptr[kSlots] = {};
    size_t slot_bytes[kSlots] = {};
    int* flags = nullptr;          // device status words (see FLAG_*)
    void* pinned = nullptr;        // small pinned host buffer for read-backs
    int lanes[5] = {4, 4, 1, 4, 1};   // lanes per particle of the float32 pair passes (SPH_PASS_*)
    int stage_cap = 0;             // most neighbour records a tile stages in shared memory (0: default)
    int tile_pipe = SPH_PIPE_GEOM;   // planned TL passes: how pair entries reach a block (SPH_PIPE_*)
    int entry_ring = SPH_RING_AUTO;  // planned Eulerian passes: how a block reads its entries (SPH_RING_*)
    bool waits_pending = false;    // a kernel with bounded waits ran since the timeout flag was read
    uint32_t wait_test_polls = 0;  // failure-detection test: bounded waits on a phase nothing completes
    double relax_skin = 0.2;       // float32 relaxation: list skin / h (0: a cell sweep every step)
    // planned TL passes: their gathered records marked persisting in L2 (sph_set_l2_persist)
    int l2_persist = 1;
    size_t l2_setaside = 0;        // the persisting set-aside this context asked for (0: none)
    size_t l2_max_window = 0;      // cudaDevAttrMaxAccessPolicyWindowSize
    // batched Eulerian step: launch shape, captured graph and the case table it was made for
    int batch_block = 256;
    cudaGraphExec_t batch_graph = nullptr;
    cudaStream_t capture_stream = nullptr;
    // second stream and events of the float32 host-state step (sph_tlsph_step_host32)
    cudaStream_t side_stream = nullptr;
    cudaEvent_t side_ev[4] = {};
    BatchGraphKey batch_key = {};
    std::vector<unsigned char> batch_blob;
};

// scratch slots (each is a grow-only device buffer owned by the context)
enum ScratchSlot {
    S_CELL_ID = 0, S_CELL_COUNT, S_CELL_START, S_CELL_FILL, S_SORTED, S_P32SORTED,
    S_ROW_LEN, S_SCAN_BLOCKS, S_ABSMAX, S_RELAX_ROWPTR, S_RELAX_COL, S_RELAX_ACC,
    S_RELAX_AMAX, S_RED_PARTIAL, S_KGC_COUNT, S_MISC0, S_MISC1, S_MISC2, S_MISC3, S_BATCH, S_MLP_PARTS,
    S_LEARN0, S_LEARN1, S_LEARN2, S_TL_VOUT
};

// device status words
enum { FLAG_BAD_INPUT = 0, FLAG_NONFINITE = 1, FLAG_CAPACITY = 2, FLAG_TIMEOUT = 3, FLAG_STALE = 4, FLAG_COUNT = 8 };

#define SPH_CUDA(ctx, call)                                                     \
    do {                                                                        \
        cudaError_t e_ = (call);                                                \
        if (e_ != cudaSuccess) {                                                \
            if (ctx) (ctx)->last_cuda_error = (int)e_;                          \
            return SPH_ERR_CUDA;                                                \
        }                                                                       \
    } while (0)

#define SPH_LAUNCH_CHECK(ctx) SPH_CUDA(ctx, cudaGetLastError())

// Programmatic dependent launch.  A kernel launched with the programmatic-serialization
// attribute may start while the previous kernel of its stream is finishing: it reads only
// data no kernel in flight writes before grid_dependency_wait(), which returns once that
// previous kernel has completed and its writes are visible; grid_launch_dependents() lets
// the next such kernel start.  Both are no-ops in a kernel launched without the attribute.
__device__ __forceinline__ void grid_dependency_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void grid_launch_dependents() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// An L2 access-policy window of one launch: accesses to [base, base + bytes) are marked
// persisting with probability hit (the rest streaming); none when bytes == 0.
struct L2Win {
    const void* base = nullptr;
    size_t bytes = 0;
    float hit = 0.0f;
};

// The window for a buffer of `bytes` at `base` that a pass gathers from, `total` the bytes
// of all buffers given windows between passes: reserves the context's persisting set-aside
// (cudaLimitPersistingL2CacheSize, up to the device's maximum) on first use and scales hit so
// that about the set-aside persists.  An empty window when the setting is off or the runtime
// refuses it.
L2Win sph_l2_window(sph_ctx* ctx, const void* base, size_t bytes, size_t total);

// Launch with the programmatic-serialization attribute (see grid_dependency_wait), or
// without it (dependent = false: an ordinary launch, e.g. after a cross-stream event wait),
// and with the access-policy window w when it is not empty.
template <typename... KArgs, typename... Args>
inline cudaError_t launch_dependent_win(bool dependent, const L2Win& w, void (*f)(KArgs...), dim3 grid, dim3 block,
                                        size_t smem, cudaStream_t s, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[2];
    unsigned na = 0;
    if (dependent) {
        at[na].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        at[na].val.programmaticStreamSerializationAllowed = 1;
        ++na;
    }
    if (w.bytes) {
        at[na].id = cudaLaunchAttributeAccessPolicyWindow;
        at[na].val.accessPolicyWindow.base_ptr = const_cast<void*>(w.base);
        at[na].val.accessPolicyWindow.num_bytes = w.bytes;
        at[na].val.accessPolicyWindow.hitRatio = w.hit;
        at[na].val.accessPolicyWindow.hitProp = cudaAccessPropertyPersisting;
        at[na].val.accessPolicyWindow.missProp = cudaAccessPropertyStreaming;
        ++na;
    }
    cfg.attrs = at;
    cfg.numAttrs = na;
    return cudaLaunchKernelEx(&cfg, f, args...);
}

template <typename... KArgs, typename... Args>
inline cudaError_t launch_dependent(bool dependent, void (*f)(KArgs...), dim3 grid, dim3 block, size_t smem,
                                    cudaStream_t s, Args... args) {
    return launch_dependent_win(dependent, L2Win{}, f, grid, block, smem, s, args...);
}

// Per-kernel timing: returns a token for sph_timer_end (or -1 when timing is off).
int sph_timer_begin(sph_ctx* ctx, int slot, cudaStream_t s);
void sph_timer_end(sph_ctx* ctx, int token, cudaStream_t s);

// Returns a device buffer of at least `bytes` for `slot` (grown, never shrunk).
void* sph_scratch(sph_ctx* ctx, int slot, size_t bytes, int* status);

static inline cudaStream_t as_stream(void* s) { return (cudaStream_t)s; }

// Host-side domain validation shared by every entry point.
int sph_check_domain(const sph_domain* dom);

// ---------------------------------------------------------------------------
// Cell grid (host side, float64, identical arithmetic to the definition)
struct CellGrid {
    int dim;
    int n[3];
    double size[3];
    double lo[3];
    double len[3];
    double half[3];
    uint32_t periodic;
    int64_t total;
    double rc2;          // (kappa h)^2
};
CellGrid sph_make_grid(const sph_domain* dom);

// ---------------------------------------------------------------------------
// Kernel functions.  Both return the factor gs with grad W_ij = gs * r_ij,
// i.e. gs = (dW/dr)/r, written without a division by r:
//   Wendland C2 (Eq. 6): gs = -5 alpha_d h^-(d+2) (1 - q/2)^3
//   Laguerre-Gauss (Eq. 8): gs = -(ahat_d h^-(d+2)/3) e^{-q^2} (9 - 5 q^2 + q^4)
#define SPH_PI 3.14159265358979323846

static inline double wendland_alpha(int dim) {
    return dim == 2 ? 7.0 / (4.0 * SPH_PI) : (dim == 3 ? 21.0 / (16.0 * SPH_PI) : 0.75);
}
static inline double lg_alpha(int dim) {
    return dim == 2 ? 6.0 / (5.0 * SPH_PI)
                    : (dim == 3 ? 8.0 / (7.0 * pow(SPH_PI, 1.5)) : 8.0 / (7.0 * sqrt(SPH_PI)));
}

template <typename R>
__device__ __forceinline__ R wendland_gs(R q, R coef) {   // coef = -5 alpha h^-(d+2)
    R t = R(1) - R(0.5) * q;
    return coef * t * t * t;
}
template <typename R>
__device__ __forceinline__ R lg_gs(R q, R coef) {          // coef = -ahat h^-(d+2) / 3
    R q2 = q * q;
    return coef * exp(-q2) * (R(9) - R(5) * q2 + q2 * q2);
}
template <>
__device__ __forceinline__ float lg_gs<float>(float q, float coef) {
    float q2 = q * q;
    return coef * expf(-q2) * (9.0f - 5.0f * q2 + q2 * q2);
}

// ---------------------------------------------------------------------------
// Compensated (Kahan) accumulator.
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float sub_rn(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double sub_rn(double a, double b) { return __dsub_rn(a, b); }

template <typename R>
struct Kahan {
    R s, c;
    __device__ __forceinline__ void init() { s = R(0); c = R(0); }
    // every step rounds on its own (no multiply-add contraction with the caller's
    // product), so a sum is the same wherever it is inlined
    __device__ __forceinline__ void add(R x) {
        R y = sub_rn(x, c);
        R t = add_rn(s, y);
        c = sub_rn(sub_rn(t, s), y);
        s = t;
    }
    __device__ __forceinline__ R value() const { return sub_rn(s, c); }
};

// Two compensated accumulators in one register pair, on Blackwell's paired
// float32 instructions (FADD2/FFMA2): the same operations as Kahan above, with the
// compensation kept negated so that every step is an add (s - t is fma(t, -1, s),
// exact negation, one rounding).
struct Kahan2 {
    float2 s, cn;
    __device__ __forceinline__ void init() { s = make_float2(0.0f, 0.0f); cn = s; }
    __device__ __forceinline__ void add(float2 x) {
        float2 y = __fadd2_rn(x, cn);
        float2 t = __fadd2_rn(s, y);
        cn = __fadd2_rn(__ffma2_rn(t, make_float2(-1.0f, -1.0f), s), y);
        s = t;
    }
    __device__ __forceinline__ float2 value() const { return __fadd2_rn(s, cn); }
};

// One 32-byte record, read with a single 256-bit load.
struct __align__(32) F8 {
    float v[8];
};

// 256-bit streaming read of data used once: not kept in L1, and the L2 fetches the
// surrounding 256 bytes (the next entries of the same stream).
__device__ __forceinline__ F8 ldg8_stream(const float* p) {
    F8 r;
    asm("ld.global.nc.L1::no_allocate.L2::256B.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
        : "=f"(r.v[0]), "=f"(r.v[1]), "=f"(r.v[2]), "=f"(r.v[3]), "=f"(r.v[4]), "=f"(r.v[5]), "=f"(r.v[6]),
          "=f"(r.v[7])
        : "l"(p));
    return r;
}

// 32-bit streaming read of data used once (as ldg8_stream).
__device__ __forceinline__ int ldg1_stream(const int* p) {
    int r;
    asm("ld.global.nc.L1::no_allocate.L2::256B.b32 %0, [%1];" : "=r"(r) : "l"(p));
    return r;
}

// 128-bit streaming read of data used once (as ldg8_stream).
__device__ __forceinline__ float4 ldg4_stream(const float4* p) {
    float4 r;
    asm("ld.global.nc.L1::no_allocate.L2::256B.v4.f32 {%0,%1,%2,%3}, [%4];"
        : "=f"(r.x), "=f"(r.y), "=f"(r.z), "=f"(r.w)
        : "l"(p));
    return r;
}

// 256-bit read-only gather (the record must not be written during the kernel).
__device__ __forceinline__ F8 ldg8(const float* p) {
    F8 r;
    asm("ld.global.nc.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
        : "=f"(r.v[0]), "=f"(r.v[1]), "=f"(r.v[2]), "=f"(r.v[3]), "=f"(r.v[4]), "=f"(r.v[5]), "=f"(r.v[6]),
          "=f"(r.v[7])
        : "l"(p));
    return r;
}

// Cell-relative float32 positions: per axis a grid of n_a cells of size S_a over the
// box, x = lo + c S + o with the integer cell c packed 10 bits per axis (3D) or 15
// (2D) into one 32-bit word, bit 30 free for a flag.  r_ij = (c_i - c_j) S + (o_i - o_j)
// keeps float32 accuracy of r itself in any box.  The grid is finer than h (up to
// kRelCellsPerH cells per h, as the bit width allows): the rounding of o_i shifts every
// pair of particle i alike, so it adds up coherently in sums such as sum_j V_j grad W_ij
// that nearly cancel, and a smaller S makes that shift small against the per-pair
// rounding of r.
constexpr double kRelCellsPerH = 16.0;

struct RelGrid {
    double lo[3], len[3], S[3];
    int n[3];
    uint32_t periodic;
};

static inline RelGrid make_rel_grid(const sph_domain& d) {
    RelGrid g;
    int nmax = d.dim == 3 ? 1023 : 32767;
    g.periodic = d.periodic_mask;
    for (int a = 0; a < 3; ++a) {
        if (a < d.dim) {
            double m = floor(kRelCellsPerH * d.len[a] / d.h);
            if (m < 1.0) m = 1.0;
            if (m > nmax) m = nmax;
            g.n[a] = (int)m;
            g.lo[a] = d.lo[a];
            g.len[a] = d.len[a];
            g.S[a] = d.len[a] / m;
        } else {
            g.n[a] = 1; g.lo[a] = 0.0; g.len[a] = 1.0; g.S[a] = 1.0;
        }
    }
    return g;
}

// The minimum image taken in cell units (|c_i - c_j| <= n/2, then |r| < len/2 + S) picks
// the true image of every pair closer than rc when len >= 2 rc + 2 S on each periodic axis:
// the other images are at least len - rc away.
static inline bool rel_grid_periodic_ok(const RelGrid& g, int dim, double rc) {
    for (int a = 0; a < dim; ++a)
        if (((g.periodic >> a) & 1u) && g.len[a] < 2.0 * rc + 2.0 * g.S[a]) return false;
    return true;
}

template <int DIM>
__device__ __forceinline__ int rel_cell_of(uint32_t bits, int a) {
    return DIM == 3 ? (int)((bits >> (10 * a)) & 1023u) : (int)((bits >> (15 * a)) & 32767u);
}

// The same cell coordinate as the float 2^23 + c: the 10 (15) bits or'ed into the
// mantissa of 2^23.  The difference of two such floats is c_i - c_j exactly, with
// no integer-to-float conversion.
template <int DIM>
__device__ __forceinline__ float rel_cell_f(uint32_t bits, int a) {
    constexpr int B = DIM == 3 ? 10 : 15;
    constexpr uint32_t M = (1u << B) - 1u;
    return __uint_as_float(((bits >> (B * a)) & M) | 0x4B000000u);
}

// Encode one position (float64 x per axis) as offsets and packed cells.
template <int DIM>
__device__ __forceinline__ uint32_t rel_encode(const double* x, const RelGrid& g, float* o) {
    uint32_t bits = 0;
    for (int a = 0; a < DIM; ++a) {
        double rel = x[a] - g.lo[a];
        double c = floor(rel / g.S[a]);
        if (((g.periodic >> a) & 1u) && c >= g.n[a]) { rel -= g.len[a]; c = floor(rel / g.S[a]); }
        if (c < 0.0) c = 0.0;
        if (c > g.n[a] - 1) c = g.n[a] - 1;
        o[a] = (float)(rel - c * g.S[a]);
        bits |= (uint32_t)c << (DIM == 3 ? 10 * a : 15 * a);
    }
    return bits;
}

// r_ij from two encoded positions; ncell per axis, cell size split S = Sh + Sl into
// two floats (so the c S part carries no float32 rounding of S, which would bias
// every pair of the same cell offset alike), minimum image in cell units.
template <int DIM, bool PER>
__device__ __forceinline__ void rel_pair(const float* oi, uint32_t bi, const float* oj, uint32_t bj,
                                         const int* ncell, const float* Sh, const float* Sl, uint32_t periodic,
                                         float* r, float& d2) {
    d2 = 0.0f;
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
        float fdc = rel_cell_f<DIM>(bi, a) - rel_cell_f<DIM>(bj, a);
        if (PER && ((periodic >> a) & 1u)) {
            float nc = (float)ncell[a];
            if (2.0f * fdc > nc) fdc -= nc;
            else if (2.0f * fdc < -nc) fdc += nc;
        }
        r[a] = fmaf(fdc, Sh[a], fmaf(fdc, Sl[a], oi[a] - oj[a]));
        d2 = fmaf(r[a], r[a], d2);
    }
}

// Plain accumulator with the same interface (float64 path).
template <typename R>
struct Plain {
    R s;
    __device__ __forceinline__ void init() { s = R(0); }
    __device__ __forceinline__ void add(R x) { s += x; }
    __device__ __forceinline__ R value() const { return s; }
};

// Sum over the LANES consecutive lanes of a group (butterfly, all lanes get it).
template <int LANES, typename R>
__device__ __forceinline__ R group_sum(R v) {
#pragma unroll
    for (int o = LANES / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// ---------------------------------------------------------------------------
// Device-wide exclusive scan of int32 counts into int64 offsets:
// out[i] = sum_{k<i} in[i] for i in [0, n], out[n] = total.
int sph_exclusive_scan_i64(sph_ctx* ctx, const int32_t* in, int64_t* out, int64_t n,
                           cudaStream_t s);
// Same into int32 offsets (the caller guarantees the total fits).
int sph_exclusive_scan_i32(sph_ctx* ctx, const int32_t* in, int32_t* out, int64_t n,
                           cudaStream_t s);
// Context-free variants with a caller-provided block-sum buffer of at least
// n / 2048 + 2 elements.
int sph_exclusive_scan_i64_buf(const int32_t* in, int64_t* out, int64_t n, int64_t* bsum, cudaStream_t s);
int sph_exclusive_scan_i32_buf(const int32_t* in, int32_t* out, int64_t n, int32_t* bsum, cudaStream_t s);

// Raises a kernel's dynamic shared-memory limit to the per-block maximum, once
// per (kernel, device); thread-safe.
void sph_allow_dynamic_smem(const void* kernel);

// Reads and clears the device timeout flag: SPH_ERR_TIMEOUT when a bounded wait of
// a kernel expired since the last call (synchronises the stream).
int sph_take_timeout(sph_ctx* ctx, cudaStream_t s);

// Grid size helper.
static inline unsigned grid_for(int64_t n, int block) {
    int64_t g = (n + block - 1) / block;
    return (unsigned)(g < 1 ? 1 : g);
}
