/*
 * sph.h -- C ABI of libsph, the GB300 (sm_103a) implementation of the
 * truncated-kernel SPH hot path of "An efficient truncation scheme for Eulerian
 * and total Lagrangian SPH methods" (arXiv 2405.05155).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Pointers: every array argument is a DEVICE pointer unless its name ends in
 *   _host.  Arrays are structure-of-arrays, component-major: a vector field of
 *   dimension d over n particles is stored as x[k*n + i], k < d.  The packed
 *   FP32 records described below are array-of-records, 16-byte aligned.
 * Ownership: the caller allocates and owns every argument array.  A context
 *   (sph_ctx) owns only internal scratch (cell lists, scan buffers, flags),
 *   grown on demand and freed by sph_destroy.
 * Streams: `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *   stream).  Calls enqueue work and return without waiting, except where a
 *   comment says the call synchronises the stream (every call that returns a
 *   value through a _host pointer does).
 * Status: every entry point returns SPH_OK (0) or one of the SPH_ERR_* codes;
 *   no call aborts, traps or prints.  sph_status_string() names a code and
 *   sph_last_cuda_error() gives the CUDA error behind SPH_ERR_CUDA.
 * Geometry: r_ij = r_i - r_j (minimum image on periodic axes: dx > L/2 -> dx-L,
 *   dx < -L/2 -> dx+L), grad W_ij = (dW/dr) r_ij/|r_ij| (the gradient with
 *   respect to r_i).  j is a neighbour of i when j != i and the float64
 *   squared distance ((dx*dx)+dy*dy)+dz*dz, every operation rounded on its own,
 *   is <= (kappa*h)*(kappa*h): the compact support of Eq. 5 (Sec. 2.2) with
 *   cut-off 2h (standard) or 1.6h (truncated, Sec. 2.3.1).
 * Symmetric 2x2 / 3x3 matrices are stored by their unique entries row by row:
 *   2D (m00, m01, m11), 3D (m00, m01, m02, m11, m12, m22): nsym = 3 or 6.
 * Full d x d matrices (F - I, stresses) are stored row-major: entry (a,b) is
 *   component a*d + b.
 */
#ifndef SPH_H
#define SPH_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define SPH_OK            0
#define SPH_ERR_ARG       1  /* bad argument: null pointer, dim not 2/3, n < 0, h <= 0,
                                kappa not in (0,2], periodic box < 2 kappa h, bad enum,
                                position not finite or outside a periodic box */
#define SPH_ERR_CAPACITY  2  /* output array too small; the required size is returned */
#define SPH_ERR_CUDA      3  /* a CUDA runtime call failed; see sph_last_cuda_error */
#define SPH_ERR_TIMEOUT   4  /* a bounded device-side wait expired */
#define SPH_ERR_NONFINITE 5  /* a reduction met a NaN or infinity */
#define SPH_ERR_LIMIT     6  /* input larger than a fixed internal limit (sph_build_neighbors_static) */

/* ---- enums ---- */
#define SPH_WENDLAND_C2     0  /* Eq. 6; cut-off kappa*h, kappa = 2 or 1.6 */
#define SPH_LAGUERRE_GAUSS  1  /* Eq. 8, normalised by ahat_d = 8/(7 sqrt(pi)),
                                  6/(5 pi), 8/(7 pi^1.5); cut-off 2h */
#define SPH_FP64            0  /* every operation in float64 */
#define SPH_FP32_KAHAN      1  /* float32 pair loops with compensated (Kahan) sums */
#define SPH_TWO_PASS        0  /* Eulerian step: momentum pass, then continuity pass */
#define SPH_FUSED           1  /* Eulerian step: one forward-Euler pass */
#define SPH_SVK             0  /* St Venant-Kirchhoff, Eq. 29 */
#define SPH_NEO_HOOKEAN     1  /* compressible neo-Hookean S = G(I - C^-1) + lambda ln J C^-1 */

#define SPH_MAX_SPHERES    16

typedef struct sph_ctx sph_ctx;

/* Particle set geometry.  dim 2 or 3; n particles; smoothing length h; cut-off
 * factor kappa (support radius kappa*h); box [lo, lo+len) per axis, used for
 * the cell grid (every axis) and the minimum image (axes whose bit is set in
 * periodic_mask).  Cells: n_k = max(1, floor(len_k/(kappa h))) per axis of size
 * len_k/n_k; particles outside the box of a non-periodic axis go to the edge
 * cell.  On a periodic axis positions must lie in [lo, lo+len] and
 * len >= 2 kappa h. */
typedef struct {
    int32_t  dim;
    uint32_t periodic_mask;
    int64_t  n;
    double   h;
    double   kappa;
    double   lo[3];
    double   len[3];
} sph_domain;

/* ---- context ---- */

/* Create a context on CUDA device `device`; *ctx receives it.  Allocates no
 * device memory until a call needs scratch. */
int sph_create(sph_ctx** ctx, int device);
/* Free the context and its scratch (synchronises the device). */
int sph_destroy(sph_ctx* ctx);
/* Static string naming a status code. */
const char* sph_status_string(int status);
/* The cudaError_t value of the most recent failed CUDA call in this context. */
int sph_last_cuda_error(const sph_ctx* ctx);

/* Host buffers the device reads and writes in place (not part of the paper: the
 * end-to-end path with host state).  sph_host_alloc allocates `bytes` of page-
 * locked host memory mapped into the device address space (cudaHostAlloc with
 * cudaHostAllocMapped | cudaHostAllocPortable) and returns the host pointer in
 * *host and the pointer device code uses in *dev.  Any array argument of the
 * entry points may be such a device pointer: the kernels then move the data over
 * the host link themselves (NVLink-C2C on Grace-Blackwell), with no separate copy.
 * sph_host_free releases a buffer of sph_host_alloc.  SPH_ERR_ARG for null
 * pointers or bytes == 0; SPH_ERR_CUDA if the runtime refuses (nothing is
 * allocated then). */
int sph_host_alloc(size_t bytes, void** host, void** dev);
int sph_host_free(void* host);

/* Launch shape of the float32 pair passes: `lanes` (1, 2, 4 or 8) consecutive
 * lanes of a warp share one particle's neighbour row (for SPH_PASS_RELAX: the
 * row of the float32 relaxation list) and combine their partial
 * sums with shuffles.  pass: SPH_PASS_*.  Results of different shapes differ
 * only by float32 rounding.  Defaults to 4 (1 for SPH_PASS_RELAX and
 * SPH_PASS_COMPRESSIBLE, the float32 pass of sph_compressible_step).  sph_get_lanes returns the setting
 * (or -1 on a bad argument).  Not part of the paper: a GPU launch parameter. */
#define SPH_PASS_EULERIAN 0
#define SPH_PASS_TLSPH    1
#define SPH_PASS_RELAX    2
#define SPH_PASS_COMPRESSIBLE 4
int sph_set_lanes(sph_ctx* ctx, int pass, int lanes);
int sph_get_lanes(const sph_ctx* ctx, int pass);
/* Most neighbour records a tile of a planned pass stages in shared memory (0: as
 * many as the plan needs, within 96 KB); tiles with more read their neighbours from
 * global memory.  A launch-shape setting, like the lanes: results do not depend on it. */
int sph_set_stage_cap(sph_ctx* ctx, int cap);
/* How the planned Eulerian passes (single and batched) read their pair entries (a
 * launch-shape setting: results do not depend on it):
 *   SPH_RING_AUTO    the chunk ring for launches of at least two waves of blocks
 *                    (2 x 6 blocks per SM x SMs), else the thread ring (the default);
 *   SPH_RING_THREAD  each thread streams its own entries through 4 slots in shared
 *                    memory with cp.async (the shorter chain when one wave is the pass);
 *   SPH_RING_CHUNK   one step of the tile's entries (4 KB) per TMA bulk copy, 4 in flight,
 *                    each completing on an mbarrier and refilled when the block has read it
 *                    (bounded waits: SPH_ERR_TIMEOUT at the next unpack).
 * SPH_ERR_ARG for any other mode. */
#define SPH_RING_AUTO   0
#define SPH_RING_THREAD 1
#define SPH_RING_CHUNK  2
int sph_set_entry_ring(sph_ctx* ctx, int mode);
/* L2 residency of the planned TL passes' gathered records (on = 1, the default): the
 * geometry-form passes launch with an access-policy window that marks the float32 records
 * they gather (rm in the momentum pass, rd in the deformation pass) persisting in L2, so
 * that they stay there from one pass and step to the next.  On first use the context
 * reserves a persisting set-aside of L2 (cudaLimitPersistingL2CacheSize: the records'
 * bytes, at most the device's maximum; with more records than that a matching fraction of
 * the accesses is marked) for the process's CUDA context on the device, which lasts until
 * sph_set_l2_persist(ctx, 0) or sph_destroy: both synchronise the device, turn the lines
 * marked persisting back to normal and set the set-aside to 0.  A launch-shape setting:
 * results do not depend on it.  SPH_ERR_ARG for on other than 0 or 1; SPH_ERR_CUDA if the
 * device synchronisation fails.  If the runtime refuses the set-aside the passes launch
 * without windows and the setting reads as off. */
int sph_set_l2_persist(sph_ctx* ctx, int on);
/* Planned TL passes, how pair entries reach a block (a launch-shape setting:
 * results do not depend on it, apart from the rounding SPH_PIPE_GEOM notes):
 *   SPH_PIPE_STREAM     one block per tile, entries streamed from global memory;
 *   SPH_PIPE_PERSISTENT one block per SM, the next tile's entries and neighbours
 *                       copied into shared memory by TMA while the current tile
 *                       computes (when its buffers fit);
 *   SPH_PIPE_BULK       one block per tile; the deformation pass copies the tile's
 *                       whole entry block into shared memory with one TMA bulk copy
 *                       while it stages the neighbours;
 *   SPH_PIPE_GEOM       one block per tile; both passes stage the neighbours'
 *                       positions (and the deformation pass their velocities, the
 *                       momentum pass V0_j M_j) and evaluate each pair's
 *                       grad0 W_ij V0_j from them, reading only the entries' 2-byte
 *                       neighbour slots; the momentum pass sums Eq. 30 as
 *                       M_i S_i + sum_j (V0_j M_j) grad0 W_ij with the plan's
 *                       S_i = sum_j grad0 W_ij V0_j (boxes with a periodic axis: the
 *                       momentum pass streams its entries); the deformation pass
 *                       copies the tile's slots into shared memory with one TMA bulk
 *                       copy (bounded wait); both passes are launched as programmatic
 *                       dependents of the pass before.  Results differ from the
 *                       other modes by float32 rounding.  The default: the fastest
 *                       measured.
 * SPH_ERR_ARG for any other mode. */
#define SPH_PIPE_STREAM     0
#define SPH_PIPE_PERSISTENT 1
#define SPH_PIPE_BULK       2
#define SPH_PIPE_GEOM       3
int sph_set_tile_pipeline(sph_ctx* ctx, int mode);
/* Failure-detection test of the bounded device waits (no counterpart in the paper).
 * polls > 0: the bounded-wait kernels of the SPH_PIPE_BULK deformation pass issue no
 * bulk copy and wait at most `polls` polls on an mbarrier phase that nothing
 * completes, so every block takes its timeout branch (sets the timeout flag, writes
 * nothing, leaves with no copy in flight) and the next sph_tlsph_unpack returns
 * SPH_ERR_TIMEOUT.  0 (default) restores normal operation.  SPH_ERR_ARG for polls
 * above 65536. */
int sph_set_wait_test(sph_ctx* ctx, uint32_t polls);

/* Per-kernel device timing (not part of the paper: measurement support).
 * sph_timing_enable(ctx, k) with k >= 1 clears the counters and makes the step
 * entry points record a CUDA event pair, on the launch stream, around every k-th
 * kernel launch of each slot (k = 1: every launch; a larger k keeps the events' own
 * cost out of a timed run); sph_timing_enable(ctx, 0) stops recording (SPH_ERR_ARG
 * for k < 0).  sph_timing_read synchronises on the recorded events and returns, for
 * one SPH_TIMER_* slot, the summed device time in milliseconds of the timed launches
 * and their number; sph_timing_launches returns all launches of the slot since
 * timing was enabled, timed or not. */
#define SPH_TIMER_TL_STRESS    0
#define SPH_TIMER_TL_MOMENTUM  1
#define SPH_TIMER_TL_DEFORM    2
#define SPH_TIMER_EU_MOMENTUM  3
#define SPH_TIMER_EU_MASS      4
#define SPH_TIMER_EU_FUSED     5
#define SPH_TIMER_NEIGHBORS    6
#define SPH_TIMER_RELAX_ACCEL  7
#define SPH_TIMER_RELAX_UPDATE 8
#define SPH_TIMER_BATCH_STEP   9  /* one replay of the captured batched step (2 launches) */
#define SPH_TIMER_SLOTS        16
int sph_timing_enable(sph_ctx* ctx, int on);
int sph_timing_read(sph_ctx* ctx, int slot, double* total_ms_host, int64_t* launches_host);
int sph_timing_launches(const sph_ctx* ctx, int slot, int64_t* launches_host);

/* ---- a3: kernel values and radial derivatives ----
 * Eq. 6 (Wendland C2, Sec. 2.3.1) or Eq. 8 (Laguerre-Gauss, Sec. 2.3.2).
 * For n distances r[i] >= 0 writes w[i] = W(r) and dwdr[i] = dW/dr, computed in
 * `precision` (results widened to float64), with the cut at q = r/h <= kappa
 * (values beyond are 0).  w or dwdr may be NULL. */
int sph_kernel_eval(int kernel, int dim, double h, double kappa, int precision,
                    const double* r, double* w, double* dwdr, int64_t n, void* stream);

/* ---- a1: cell binning and order ----
 * Sec. 2.3 (cell-linked lists).  Permutation order[k] (int64, length n) sorting the
 * particles by (Morton key of the cell, original index), stable.  The cell is
 * c_k = floor((x_k - lo_k)/size_k) with n_k = max(1, floor(len_k/(kappa h))) cells
 * of size len_k/n_k per axis, wrapped on periodic axes and clamped otherwise.  The
 * Morton key interleaves the coordinate bits level by level from the least
 * significant, axes in order x, y, z; an axis with ceil(log2 n_k) bits drops out once
 * they are used.  Particles consecutive in this order form compact groups, which the
 * pair passes stage in shared memory.  pos: float64 [dim][n].  SPH_ERR_ARG when the
 * key needs more than 29 bits or a position is non-finite (or outside a periodic box).
 * Synchronises the stream (to validate positions). */
int sph_cell_order(sph_ctx* ctx, const sph_domain* dom, const double* pos,
                   int64_t* order, void* stream);

/* ---- a2: CSR neighbour lists ----
 * Compact-support neighbour sets of Eq. 5 with cut-off kappa*h: row i holds
 * every j != i with float64 d^2 <= (kappa h)^2 (see the header comment), sorted
 * ascending.  pos float64 [dim][n]; row_ptr int64 [n+1]; col int32 [cap].
 * *nnz_host receives row_ptr[n].  If cap < nnz nothing is written to col and
 * SPH_ERR_CAPACITY is returned with *nnz_host = the required capacity
 * (row_ptr is valid).  Synchronises the stream once, to read nnz; the fill of
 * col is then enqueued on `stream` and is complete when the stream reaches it
 * (row_ptr and *nnz_host are final on return).  Bit-exact with the float64
 * definition: candidates are screened in float32 with a proven error band and
 * every candidate inside the band is decided in float64. */
int sph_build_neighbors(sph_ctx* ctx, const sph_domain* dom, const double* pos,
                        int64_t* row_ptr, int32_t* col, int64_t cap,
                        int64_t* nnz_host, void* stream);

/* ---- allocation-free neighbour lists ----
 * The paper has no counterpart: this is a deployment variant of
 * sph_build_neighbors for callers that cannot allocate device memory, such as a
 * plug-in inside an application that owns the whole device-memory budget (it
 * reserves its pool at start-up and treats any other cudaMalloc as a failure),
 * or a latency-critical loop in which cudaMalloc/cudaFree would synchronise the
 * device.  Same arguments, results and status codes as sph_build_neighbors, but
 * no context and no allocation of any kind: all internal scratch lives in one
 * static device array of SPH_STATIC_SCRATCH_BYTES (44 MiB) that every GPU
 * loading libsph holds until the process exits.  The caller provides pos,
 * row_ptr and col as usual.  Limits: n <= SPH_STATIC_MAX_PARTICLES and at most
 * SPH_STATIC_MAX_CELLS cells in the grid (n_x n_y n_z of the sph_domain comment);
 * larger inputs return SPH_ERR_LIMIT before any device work.  Every call looks
 * up the array's device address on the current device (cudaGetSymbolAddress, a
 * host-side lookup that the first call on a device also uses to load the
 * module), so make the first call on each device before any stream capture.
 * Every call reuses the same array and clears what must start at zero; calls
 * that overlap on the GPU (from two streams or two host threads) race on it and
 * must be serialised by the caller.  Synchronises the stream once, to read nnz;
 * the fill of col is then enqueued on `stream` and is complete when the stream
 * reaches it.  On SPH_ERR_CUDA the CUDA error is left for cudaGetLastError()
 * (this call only peeks at it). */
#define SPH_STATIC_MAX_PARTICLES (1 << 20)
#define SPH_STATIC_MAX_CELLS     (1 << 20)
#define SPH_STATIC_SCRATCH_BYTES (44u << 20)
int sph_build_neighbors_static(const sph_domain* dom, const double* pos,
                               int64_t* row_ptr, int32_t* col, int64_t cap,
                               int64_t* nnz_host, void* stream);

/* ---- a4: kernel gradient correction ----
 * Eq. 9 (Sec. 2.3.2): A_i = -sum_j V_j r_ij (x) grad W_ij over the CSR row,
 * B_i = A_i^-1 (adjugate formula), all float64, kernel `kernel` with the cut-off
 * of dom->kappa.  B: float64 [nsym][n].  A particle whose A_i is not finite, has
 * trace <= 0 or det A <= 1e-8 (tr A/d)^d gets B_i = I and fallback[i] = 1
 * (else 0); fallback may be NULL.  If n_fallback_host is not NULL it receives
 * the number of such particles and the call synchronises the stream. */
int sph_kgc(sph_ctx* ctx, const sph_domain* dom, int kernel, const double* pos,
            const double* vol, const int64_t* row_ptr, const int32_t* col,
            double* B, uint8_t* fallback, int64_t* n_fallback_host, void* stream);

/* ---- a5/a6: Eulerian weakly-compressible SPH (Sec. 3.1) ----
 * Fixed particles with volume V_i, density rho0 + drho_i, velocity v_i and
 * pressure p = c0^2 drho (Sec. 3.1.1).  Rates (Eq. 18 divided by w_i):
 *   d rho_i/dt      = -2 sum_j V_j rho* (v* . g)
 *   d (rho v)_i/dt  = -2 sum_j V_j [rho* v* (v* . g) + p* g]
 *                     + 2 mu sum_j V_j (v_i - v_j)(r_ij . grad W_ij)/(r^2 + 0.01 h^2)
 * with g = (B_i + B_j)/2 grad W_ij (Eq. 27, Wendland with cut-off dom.kappa),
 * normal n = -r_ij/r, u_l = v_i.n, u_r = v_j.n, rho* = (rho_i+rho_j)/2,
 * beta = min(eta max((u_l-u_r)/c0, 0), 1), u* = (u_l+u_r)/2 + beta^2 (p_i-p_j)/(2 rho* c0),
 * p* = (p_i+p_j)/2 + beta rho* c0 (u_l-u_r)/2 (Eqs. 25-26), v* = (v_i+v_j)/2 + (u* - (u_l+u_r)/2) n.
 * Time step (integrator SPH_TWO_PASS): momentum pass from (rho^n, v^n) gives
 * (rho v)^{n+1} and v' = (rho v)^{n+1}/rho^n; continuity pass from (rho^n, v')
 * gives rho^{n+1}; v^{n+1} = (rho v)^{n+1}/rho^{n+1}.  SPH_FUSED evaluates both
 * rates at (rho^n, v^n). */
typedef struct {
    sph_domain dom;
    double dt, rho0, c0, mu, eta;   /* eta = 15 in the paper (Eq. 26) */
    int32_t precision;              /* SPH_FP64 or SPH_FP32_KAHAN */
    int32_t integrator;             /* SPH_TWO_PASS or SPH_FUSED */
} sph_eulerian_params;

/* State arrays.  FP64 steps use pos/vol/B/drho/v and the drho_tmp/v_tmp
 * scratch (same shapes as drho/v).  FP32 steps use packed records of 16 floats
 * (two 32-byte lines; rec and rec_tmp 32-byte aligned), made by
 * sph_eulerian_pack from the FP64 arrays and read back by sph_eulerian_unpack:
 *   3D: (ox, oy, oz, cell, V, B00, B01, B02) (B11, B12, B22, 0, vx, vy, vz, drho)
 *   2D: (ox, oy, cell, V, B00, B01, B11, 0) (0, 0, 0, 0, vx, vy, 0, drho)
 * with the cell-relative position of the sph_tlsph_state comment (grid of
 * n_a = min(max(1, floor(len_a/h)), 1023 or 32767) cells, at least 4 along a
 * periodic axis).  Both buffers hold the static part; a pass writes only the
 * (v, drho) float4 of the other buffer. */
typedef struct {
    const int64_t* row_ptr;
    const int32_t* col;
    const double*  pos;
    const double*  vol;
    const double*  B;
    double* drho;
    double* v;
    double* drho_tmp;
    double* v_tmp;
    float*  rec;
    float*  rec_tmp;
    void*   plan;          /* optional tile plan buffer (see sph_eulerian_plan) */
    int64_t plan_bytes;
    int64_t plan_nnz;      /* written by sph_eulerian_plan */
    int32_t plan_maxm;     /* written by sph_eulerian_plan */
    int32_t plan_maxrow;   /* written by sph_eulerian_plan */
} sph_eulerian_state;

/* float64 (pos, vol, B, drho, v) -> packed float32 records (rec, rec_tmp). */
int sph_eulerian_pack(sph_ctx* ctx, const sph_eulerian_params* prm,
                      const sph_eulerian_state* st, void* stream);
/* Tile plan of the float32 passes (not an operation of the paper: a staging
 * layout of the pair pass of Eq. 18).  Eulerian particles are fixed, so the pair
 * geometry is too: sph_eulerian_plan builds in st->plan (caller-owned device
 * buffer of plan_bytes >= sph_eulerian_plan_bytes(...) bytes, 32-byte aligned),
 * from pos/vol/B/row_ptr/col and the parameters mu, h, per tile of 128 consecutive
 * rows, the list of its distinct neighbours and, per pair, in float64 then stored
 * in float32, the corrected gradient G = -2 V_j (B_i + B_j)/2 grad W_ij (Eq. 27),
 * the viscous factor 2 mu V_j (r_ij . grad W_ij)/(r^2 + 0.01 h^2), the normal
 * -r_ij/r and the neighbour's position in its tile's list, in the sliced order of
 * sph_tlsph_state.  It writes plan_nnz, plan_maxm and plan_maxrow.  The float32
 * passes then stage each tile's neighbour (v_j, drho_j) in shared memory, one
 * thread per row (the lanes setting unused).  Rebuild it when the lists, pos, vol,
 * B, h or mu change.  Synchronises the stream; SPH_ERR_CAPACITY when plan_bytes is
 * too small.  plan = NULL or plan_nnz = 0: the float32 passes evaluate the geometry
 * per pair from the records. */
int sph_eulerian_plan_bytes(sph_ctx* ctx, const sph_eulerian_params* prm, const sph_eulerian_state* st,
                            int64_t* bytes_host, void* stream);
int sph_eulerian_plan(sph_ctx* ctx, const sph_eulerian_params* prm, sph_eulerian_state* st, void* stream);
/* The weakly-compressible equation of state of Sec. 3.1.1, p = c0^2 (rho - rho0),
 * inverted for the stored density offset: drho[i] = p[i] / c0^2 for i < prm->dom.n
 * (p, drho float64 device arrays [n]; only dom.n and c0 of prm are read).  For initial
 * conditions given as a pressure field.  SPH_ERR_ARG when c0 <= 0 or a pointer is NULL
 * with n > 0. */
int sph_eulerian_density_from_pressure(sph_ctx* ctx, const sph_eulerian_params* prm, const double* p,
                                       double* drho, void* stream);
/* packed float32 rec -> float64 (drho, v). */
int sph_eulerian_unpack(sph_ctx* ctx, const sph_eulerian_params* prm,
                        const sph_eulerian_state* st, void* stream);
/* Both rates at the current state (FP64 arrays or, for FP32, the packed rec):
 * drho_dt float64 [n], dmom_dt float64 [dim][n]. */
int sph_eulerian_rates(sph_ctx* ctx, const sph_eulerian_params* prm,
                       const sph_eulerian_state* st, double* drho_dt,
                       double* dmom_dt, void* stream);
/* Advance nsteps time steps in place (drho/v for FP64, q for FP32). */
int sph_eulerian_step(sph_ctx* ctx, const sph_eulerian_params* prm,
                      const sph_eulerian_state* st, int nsteps, void* stream);
/* Autotuner of the float32 passes (not in the paper: a launch parameter): times
 * trial_steps steps of the caller's float32 state for lanes per particle in
 * {1, 2, 4, 8}, restores q after every trial, stores the fastest setting in the
 * context (SPH_PASS_EULERIAN) and returns it with its ms per step (outputs may be
 * NULL).  Synchronises the stream. */
int sph_autotune_eulerian(sph_ctx* ctx, const sph_eulerian_params* prm,
                          const sph_eulerian_state* st, int trial_steps, int* lanes_host,
                          double* ms_host, void* stream);

/* ---- a13: batched Eulerian step (not in the paper: many cases per launch) ----
 * ncases independent Eulerian cases (the float32 two-pass step of
 * sph_eulerian_step, Sec. 3.1) whose packed records and CSR lists are
 * concatenated: case c owns particles [offset, offset + n) of rec/rec_tmp, its
 * CSR rows are rows offset..offset+n-1 of row_ptr and its column indices are
 * global (already shifted by offset).  One persistent launch per pass covers
 * all cases; the two launches of a step are captured into a CUDA graph once and
 * replayed (the graph is recaptured when the buffers, case table or launch
 * shape change).  Results match sph_eulerian_step on each case alone (to float32
 * rounding: the two kernels may contract multiply-adds differently).
 * cases_host is a host array of ncases (<= 256) entries, offsets contiguous
 * from 0.  The launch shape is the context's SPH_PASS_BATCHED lanes and batch
 * block size, chosen by sph_autotune_batched. */
#define SPH_PASS_BATCHED 3
typedef struct {
    int64_t offset, n;
    int32_t dim;
    uint32_t periodic_mask;
    double h, dt, rho0, c0, mu, eta;
    double len[3];                  /* box lengths (minimum image on periodic axes) */
    /* optional: the case's tile plan (sph_eulerian_plan of the case alone, with
     * case-local indices) and the three fields that call wrote.  When every case has
     * one, the step runs the planned form: one block per tile of any case, the lanes
     * and block settings unused. */
    const void* plan;
    int64_t plan_nnz;
    int32_t plan_maxm, plan_maxrow;
} sph_batch_case;
typedef struct {
    const int64_t* row_ptr;         /* [N+1] */
    const int32_t* col;             /* global indices */
    float* rec;                     /* [N][16] records, sph_eulerian_state layout */
    float* rec_tmp;                 /* [N][16] second buffer (static part filled) */
} sph_batch_state;
int sph_eulerian_step_batched(sph_ctx* ctx, const sph_batch_case* cases_host, int ncases,
                              const sph_batch_state* st, int nsteps, void* stream);
/* Autotuner: times trial_steps steps for every launch shape (lanes per particle in
 * {1, 2, 4, 8} x block size in {128, 256}) on the caller's data, restores the state
 * after each trial, keeps the fastest shape in the context and returns it
 * (lanes, block, ms per step; any output pointer may be NULL).  Synchronises. */
int sph_autotune_batched(sph_ctx* ctx, const sph_batch_case* cases_host, int ncases,
                         const sph_batch_state* st, int trial_steps, int* lanes_host,
                         int* block_host, double* ms_host, void* stream);

/* ---- a7-a9: total-Lagrangian SPH for solids (Sec. 3.2) ----
 * Reference configuration r0 with volumes V0, correction B0 (Eq. 9 at r0) and
 * the CSR lists built at r0.  Per step: M_i = P(F_i) B0_i^T with P = F S
 * (Eq. 29 or neo-Hookean), a_i = (1/rho0) sum_j (M_i + M_j) grad0 W_ij V0_j
 * (Eq. 30), v += dt a, dF_i/dt = (sum_j V0_j (v_j - v_i) (x) grad0 W_ij) B0_i
 * (Eq. 31), F += dt dF/dt, x += dt v.  Clamped particles (fixed[i] != 0) keep
 * v = 0 and F = I. */
typedef struct {
    sph_domain dom;                 /* geometry of r0 (h, kappa, box) */
    double dt, rho0, lambda, G;
    int32_t law;                    /* SPH_SVK or SPH_NEO_HOOKEAN */
    int32_t precision;              /* SPH_FP64 or SPH_FP32_KAHAN */
} sph_tlsph_params;

/* FP64 arrays: x, v [dim][n]; H = F - I [dim*dim][n]; M scratch [dim*dim][n].
 * FP32 packed records (made by sph_tlsph_pack; rd and rm 32-byte aligned):
 *   rd [n][8]:  3D (ox, oy, oz, cell, vx, vy, vz, V0); 2D (ox, oy, cell, V0, vx, vy, 0, 0)
 *   rm [n][16]: 3D (ox, oy, oz, cell, M00, M10, M20, V0, M01, M11, M21, 0, M02, M12, M22, 0)
 *   rm [n][8]:  2D (ox, oy, cell, V0, M00, M10, M01, M11)
 *   with M = P B0^T and a cell-relative position: per axis a grid of
 *   n_a = min(max(1, floor(16 len_a/h)), 1023 (3D) or 32767 (2D)) cells of size
 *   S_a = len_a/n_a, integer cell c_a packed into `cell` (10 or 15 bits per axis,
 *   bit 30 set on clamped particles) and float offset o_a = x_a - lo_a - c_a S_a;
 *   H32 [dim*dim][n], u32 [dim][n] (x - r0), B32 [nsym][n].
 *   The float32 path needs len_a >= 2 kappa h + 2 S_a along a periodic axis.
 * Tile plan (optional, float32 path): plan -> caller-owned device buffer of
 *   plan_bytes >= sph_tlsph_plan_bytes(...) bytes, 32-byte aligned.  sph_tlsph_plan
 *   builds in it, from row_ptr/col/r0/V0, (i) per tile of 128
 *   consecutive rows the list of its distinct neighbours and (ii) per pair the
 *   reference-configuration factor w_ij = grad0 W_ij V0_j of Eqs. 30-31, computed in
 *   float64 and stored in float32 with the neighbour's position in its tile's list,
 *   in a sliced order (pair k of row r of a tile at k*128 + r).  It writes plan_nnz,
 *   plan_maxm (most distinct neighbours of a tile) and plan_maxrow (longest row)
 *   into the struct.  The pair passes then stage each tile's neighbour M_j or
 *   v_j in shared memory and read the pair factors from the plan: one thread per
 *   row, the context's lanes setting unused.  Rows are best in sph_cell_order
 *   (Morton) order, so that a tile is a compact group.  The plan must be rebuilt
 *   (sph_tlsph_plan) whenever row_ptr, col, r0 or V0 change.  plan = NULL or
 *   plan_nnz = 0 (no plan built): the pair factors are evaluated per pair from the
 *   records and neighbours are gathered from global memory. */
typedef struct {
    const int64_t* row_ptr;
    const int32_t* col;
    const double*  r0;
    const double*  V0;
    const double*  B0;
    const uint8_t* fixed;
    double* x;
    double* v;
    double* H;
    double* M;
    float*  rd;
    float*  rm;
    float*  H32;
    float*  u32;
    float*  B32;
    void*   plan;          /* optional tile plan buffer (see above) */
    int64_t plan_bytes;
    int64_t plan_nnz;      /* written by sph_tlsph_plan */
    int32_t plan_maxm;     /* written by sph_tlsph_plan */
    int32_t plan_maxrow;   /* written by sph_tlsph_plan */
} sph_tlsph_state;

/* float64 state (x, v, H, r0, V0, B0, fixed) -> float32 records. */
int sph_tlsph_pack(sph_ctx* ctx, const sph_tlsph_params* prm,
                   const sph_tlsph_state* st, void* stream);
/* Builds the tile plan in st->plan (see above) and writes plan_nnz, plan_maxm and
 * plan_maxrow.  Not an operation of the paper: a staging layout of the pair passes
 * of Eqs. 30-31.  Synchronises the stream.  SPH_ERR_ARG without st->plan,
 * SPH_ERR_CAPACITY when plan_bytes is too small. */
int sph_tlsph_plan(sph_ctx* ctx, const sph_tlsph_params* prm, sph_tlsph_state* st, void* stream);
/* Bytes of the tile-plan buffer for the state's lists (reads row_ptr; synchronises
 * the stream). */
int sph_tlsph_plan_bytes(sph_ctx* ctx, const sph_tlsph_params* prm, const sph_tlsph_state* st,
                         int64_t* bytes_host, void* stream);
/* packed float32 (rd, H32, u32) -> float64 (v, H, x = r0 + u).  After steps of
 * the planned forms with bounded waits (persistent, bulk, and the geometry form's slot
 * copy; sph_set_tile_pipeline) it synchronises the stream and
 * returns SPH_ERR_TIMEOUT if a bounded device wait expired since the previous unpack
 * (the results are then not valid). */
int sph_tlsph_unpack(sph_ctx* ctx, const sph_tlsph_params* prm,
                     const sph_tlsph_state* st, void* stream);
/* The float32 form's own dynamic state in float32, for callers that keep it outside
 * the device between steps: u = x - r0 [dim][n], v [dim][n], H = F - I [dim*dim][n]
 * (device pointers, or mapped host memory of sph_host_alloc, read or written in place).
 * sph_tlsph_load32 replaces the state of the float32 records (after one
 * sph_tlsph_pack, which also sets their fixed part); sph_tlsph_store32 copies it out.
 * The float32 step keeps exactly these values, so a load32 / step / store32 round trip
 * loses nothing against the device-resident state (half the bytes of the float64
 * pack/unpack pair). */
int sph_tlsph_load32(sph_ctx* ctx, const sph_tlsph_params* prm, const sph_tlsph_state* st,
                     const float* u, const float* v, const float* H, void* stream);
int sph_tlsph_store32(sph_ctx* ctx, const sph_tlsph_params* prm, const sph_tlsph_state* st,
                      float* u, float* v, float* H, void* stream);
/* nsteps float32 steps (Eqs. 30-31, as sph_tlsph_step) with the state kept by the caller
 * in u, v, H (the arrays of sph_tlsph_load32, device or mapped host memory): each step
 * reads the state in and writes it back, with the same values as sph_tlsph_load32,
 * sph_tlsph_step(1) and sph_tlsph_store32 in turn.  The copies overlap the passes where
 * the step allows: u is copied in by a copy engine on a second stream of the context
 * while the momentum pass runs and v copied back (from a device buffer of the context)
 * while the deformation pass runs; the stress factors are formed by the kernel that
 * reads H, and the geometry form of the deformation pass (the default on a tile plan)
 * writes H and u back itself, beside the device records.  u and v must be pinned (sph_host_alloc) or device memory.  Everything is enqueued on `stream` (which waits for the
 * second stream before returning); u, v, H must not be touched until it completes.
 * Requires precision SPH_FP32_KAHAN and the float32 records (one sph_tlsph_pack first);
 * SPH_ERR_ARG otherwise.  The call does not wait for the device: a bounded wait that
 * expires in a pass (the geometry form's slot copy) sets the context's timeout flag, which
 * sph_take_status or the next sph_tlsph_unpack reports (u, v, H are then not valid). */
int sph_tlsph_step_host32(sph_ctx* ctx, const sph_tlsph_params* prm, const sph_tlsph_state* st,
                          float* u, float* v, float* H, int nsteps, void* stream);
/* Energies of the float64 state (v, H; after float32 steps call sph_tlsph_unpack
 * first): out_host[0] = kinetic sum_i rho0 V0_i |v_i|^2 / 2, out_host[1] = stored
 * sum_i V0_i psi(F_i) with the law's stored-energy density (the potential of the
 * stress of Sec. 3.2: SVK psi = lambda/2 (tr E)^2 + G E:E, neo-Hookean
 * psi = G/2 (tr C - d) - G ln J + lambda/2 (ln J)^2).  Reduced in float64 in a fixed
 * order (deterministic).  Synchronises the stream; SPH_ERR_NONFINITE when a sum is
 * not finite. */
int sph_tlsph_energy(sph_ctx* ctx, const sph_tlsph_params* prm, const sph_tlsph_state* st,
                     double* out_host, void* stream);
/* Rates at the current state: dvdt float64 [dim][n] (Eq. 30 / rho0) and
 * dFdt float64 [dim*dim][n] (Eq. 31 with the current v). */
int sph_tlsph_rates(sph_ctx* ctx, const sph_tlsph_params* prm,
                    const sph_tlsph_state* st, double* dvdt, double* dFdt, void* stream);
int sph_tlsph_step(sph_ctx* ctx, const sph_tlsph_params* prm,
                   const sph_tlsph_state* st, int nsteps, void* stream);
/* Autotuner of the float32 passes, as sph_autotune_eulerian (rd, rm, H32 and u32
 * are restored after every trial; setting stored as SPH_PASS_TLSPH). */
int sph_autotune_tlsph(sph_ctx* ctx, const sph_tlsph_params* prm, const sph_tlsph_state* st,
                       int trial_steps, int* lanes_host, double* ms_host, void* stream);

/* ---- a10/a11: Laguerre-Gauss particle relaxation (Sec. 2.3.2, Eqs. 7-8) ----
 * dim 2 or 3.  Body = union of n_spheres spheres (cx, cy, cz, r) given by value
 * (2D: circles (cx, cy, unused, r)), signed distance phi = min_k(|x-c_k| - r_k),
 * normal grad phi of the first minimising sphere.  Per step: neighbour sets
 * (cut-off kappa h) from the current positions;
 * a_i = -(2 p0/rho)(sum_j grad W_ij V_j + I(max(-phi_i,0)) grad phi_i), W the
 * Laguerre-Gauss kernel (kappa = 2) or, for the Wendland-relaxed distributions of
 * Sec. 2.3.3, the Wendland kernel, with the surface integral over the support
 * beyond the tangent line or plane at distance d,
 *   3D: I(d) = 2 pi int_d^{kappa h} z (W(z) - W(kappa h)) dz,
 *   2D: I(d) = 2 int_0^Y (W(sqrt(d^2 + y^2)) - W(kappa h)) dy, Y = sqrt((kappa h)^2 - d^2)
 * (closed form for the 3D Laguerre-Gauss kernel, a 48-node Gauss-Legendre rule
 * otherwise); dt = 0.25 sqrt(h / max|a|); x += a dt^2/2; then particles with
 * phi > -dp/2 are moved along grad phi to phi = -dp/2.  SPH_FP32_KAHAN: 3D
 * Laguerre-Gauss only (SPH_ERR_ARG otherwise). */
typedef struct {
    sph_domain dom;                 /* dim 2 or 3, h, kappa (2 for Laguerre-Gauss), cell box */
    double dp, p0, rho;
    int32_t kernel;                 /* SPH_LAGUERRE_GAUSS or SPH_WENDLAND_C2 */
    int32_t precision;              /* SPH_FP64 or SPH_FP32_KAHAN (pair sums) */
    int32_t n_spheres;              /* 1..SPH_MAX_SPHERES */
    int32_t reserved;
    double spheres[4 * SPH_MAX_SPHERES];
} sph_relax_params;

/* Advance nsteps relaxation steps of pos (float64 [dim][n], in place).
 * SPH_FP32_KAHAN keeps, within one call, a neighbour list of cut-off 2h + skin
 * (sph_set_relax_skin) and rebuilds it only when twice the largest displacement
 * since its build exceeds the skin; every step still decides each listed pair at
 * 2h exactly, so the pair sets are those of a fresh list.  The list lives in the
 * context; each call builds it anew from pos.  Synchronises the stream every few
 * steps (to read the list's status) and at the end.  SPH_ERR_CAPACITY if a
 * particle has 65,536 or more neighbours within 2h + skin. */
int sph_relax_step(sph_ctx* ctx, const sph_relax_params* prm, double* pos,
                   const double* vol, int nsteps, void* stream);
/* Skin of the float32 relaxation list in units of h, 0 <= skin_over_h <= 1
 * (default 0.2).  0 sweeps the cells afresh every step (no list).  Not part of
 * the paper: results differ only by float32 summation order. */
int sph_set_relax_skin(sph_ctx* ctx, double skin_over_h);
/* Acceleration a (float64 [3][n]) at the current positions (one neighbour
 * build + pair pass). */
int sph_relax_accel(sph_ctx* ctx, const sph_relax_params* prm, const double* pos,
                    const double* vol, double* acc, void* stream);
/* The residual out_host[0] of sph_relax_residual (Laguerre-Gauss) from float32 pair
 * sums: one float32 acceleration evaluation (the cell sweep of SPH_FP32_KAHAN, with
 * compensated sums) gives sum_j grad W_ij V_j = -a_i rho/(2 p0) for every particle with
 * phi < -2h, where the surface term of Eq. 7 vanishes; h^2 |.|^2 and the count are reduced
 * in float64 in a fixed order.  out_host[1] = NaN (the truncated-kernel residual is not
 * formed), out_host[2] = the count.  3D, Laguerre-Gauss kernel.  Synchronises the stream. */
int sph_relax_residual_fp32(sph_ctx* ctx, const sph_relax_params* prm, const double* pos,
                            const double* vol, double* out_host, void* stream);
/* Relaxation residual over particles with phi < -2h:
 * out_host[0] = sqrt(mean |h sum_j grad W^LG_ij V_j|^2),
 * out_host[1] = the same with the truncated Wendland kernel (cut-off 1.6h),
 * out_host[2] = number of such particles.  Float64, deterministic.
 * Synchronises the stream. */
int sph_relax_residual(sph_ctx* ctx, const sph_relax_params* prm, const double* pos,
                       const double* vol, double* out_host, void* stream);

/* ---- x2: compressible Riemann SPH (Sec. 3.1, Eqs. 15-24) ----
 * Eulerian particles (fixed positions, volumes V_i) carry the conserved rho, rho v and
 * E = rho |v|^2/2 + rho e of an ideal gas, p = (gamma - 1) rho e, c^2 = gamma p/rho.
 * Eq. 18 divided by V_i, with g_ij = (B_i + B_j)/2 grad W_ij (Eq. 27, Wendland kernel
 * cut at dom.kappa, B of sph_kgc):
 *   d rho_i/dt     = -2 sum_j V_j rho_s (v_s . g_ij)
 *   d(rho v)_i/dt  = -2 sum_j V_j [rho_s v_s (v_s . g_ij) + p_s g_ij]
 *   dE_i/dt        = -2 sum_j V_j (E_s + p_s) (v_s . g_ij)
 * where (rho_s, v_s, E_s, p_s) is the interface state of the HLLC solver with the
 * dissipation limiter along n = -e_ij (left = i):
 *   S_l = u_l - c_l, S_r = u_r + c_r, beta = min(eta max((u_l - u_r)/c_bar, 0), 1),
 *   u* = (rho_l c_l u_l + rho_r c_r u_r + beta^2 (p_l - p_r))/(rho_l c_l + rho_r c_r),
 *   p* = (p_l + p_r)/2 + beta [rho_r c_r (u* - u_r) + rho_l c_l (u_l - u*)]/2,
 *   v* = u* n + (v_l + v_r)/2 - (u_l + u_r) n/2,
 *   rho*_k = rho_k (S_k - u_k)/(S_k - u*), E*_k = ((S_k - u_k) E_k - p_k u_k + p* u*)/(S_k - u*);
 * the left (right) state when S_l >= 0 and S_r > 0 (S_r <= 0 and S_l < 0), else the left
 * star (u* > 0), the right star (u* < 0) or their mean (u* = 0).  The paper prints |v|
 * in rho* and E*, and a minus in the limited p*: the normal velocity and the plus of the
 * unlimited HLLC p* are used (both needed for the pairwise antisymmetry that conserves
 * mass, momentum and energy).  Time integration: forward Euler with the fixed dt.
 * Minimum image on periodic axes.
 * precision SPH_FP64: everything in float64, the pair geometry evaluated per pair.
 * precision SPH_FP32_KAHAN: the state stays float64 (advanced in float64 by the float32
 * rates); per step the neighbours' (rho, v, p, c, E) are read as float32 records, the
 * solver runs in float32 and the row sums are compensated; the pair geometry comes from
 * the plan (sph_compressible_plan), which the state must carry. */
typedef struct {
    sph_domain dom;
    double dt, gamma, eta;          /* gamma = 1.4 and eta = 1 in the paper */
    int32_t precision;              /* SPH_FP64 or SPH_FP32_KAHAN */
    int32_t reserved;
} sph_compressible_params;

typedef struct {
    const int64_t* row_ptr;         /* CSR lists of sph_build_neighbors */
    const int32_t* col;
    const double* pos;              /* [dim][n] */
    const double* vol;              /* [n] */
    const double* B;                /* [d(d+1)/2][n], sph_kgc */
    double* rho;                    /* [n], advanced in place by sph_compressible_step */
    double* mom;                    /* [dim][n] */
    double* E;                      /* [n] */
    void* plan;                     /* SPH_FP32_KAHAN: caller-owned device buffer, 16-byte aligned */
    int64_t plan_bytes;             /* >= sph_compressible_plan_bytes(...) */
    int32_t plan_width;             /* written by sph_compressible_plan: longest row */
    int32_t reserved;
} sph_compressible_state;

/* Pair geometry of the float32 form (a layout, not an operation of the paper):
 * particles are fixed, so sph_compressible_plan computes once, in float64 from pos, vol,
 * B and the lists, per pair G_ij = -2 V_j (B_i + B_j)/2 grad W_ij and n = -r_ij/r, stores
 * them rounded to float32 with the neighbour index, pair k of row i at entry
 * (i/32)*32*W + 32k + i%32 (W = longest row), and writes plan_width = W.  Rebuild it when
 * the lists, pos, vol, B or h change (a plan of other lists gives wrong results; rows
 * longer than its width are cut, never read past).  Both calls synchronise the stream;
 * SPH_ERR_CAPACITY when plan_bytes is too small. */
int sph_compressible_plan_bytes(sph_ctx* ctx, const sph_compressible_params* prm,
                                const sph_compressible_state* st, int64_t* bytes_host, void* stream);
int sph_compressible_plan(sph_ctx* ctx, const sph_compressible_params* prm, sph_compressible_state* st,
                          void* stream);

/* Rates of Eq. 18 at the current state: drho [n], dmom [dim][n], dE [n]. */
int sph_compressible_rates(sph_ctx* ctx, const sph_compressible_params* prm,
                           const sph_compressible_state* st, double* drho, double* dmom,
                           double* dE, void* stream);
/* nsteps forward-Euler steps of (rho, rho v, E) in place. */
int sph_compressible_step(sph_ctx* ctx, const sph_compressible_params* prm,
                          const sph_compressible_state* st, int nsteps, void* stream);

/* ---- x1: SPH approximations for the error analysis (Sec. 2.3.3) ----
 * For a field f (float64 [n]) on the particles, over the pairs of CSR lists of
 * sph_build_neighbors at dom->kappa and with the kernel `kernel`
 * (SPH_WENDLAND_C2 or SPH_LAGUERRE_GAUSS):
 *   sum[i]        = sum_j f_j W_ij V_j + f_i W(0) V_i       the kernel summation;
 *                   for f = 1 the normalisation condition, Eq. 3 (Table 1);
 *   grad[a*n + i] = sum_j (f_i + f_j) (B_i grad W_ij)_a V_j  the weak form of Eq. 4 with
 *                   grad W_ij = grad_i W, with the correction matrix of Eq. 9 (B in
 *                   sph_kgc's layout) or, when B is NULL, B_i = I.
 * Either output may be NULL (then it is not computed).  Minimum image on the
 * periodic axes.  Float64. */
int sph_field_approx(sph_ctx* ctx, const sph_domain* dom, int kernel, const double* pos,
                     const double* vol, const int64_t* row_ptr, const int32_t* col,
                     const double* B, const double* f, double* sum, double* grad, void* stream);

/* ---- a12: learned relaxation proposal (not in the paper) ----
 * A 128 -> 128 -> 128 -> 128 -> 3 multilayer perceptron with GELU (erf form)
 * after each hidden layer predicts a particle's displacement / h from its
 * features.  Parameters are one float32 array of SPH_MLP_NPARAM values in the
 * order W1 [128][128] (out x in), b1 [128], W2, b2, W3, b3, W4 [3][128], b4 [3];
 * the dense layers run on BF16 tensor cores (operands rounded to bfloat16,
 * float32 accumulation).  Features (float32 [n][128]): the offsets
 * (x_j - x_i)/h of the 32 nearest neighbours within the Laguerre-Gauss support
 * 2h, ordered by (float64 squared distance, j), zero-filled, then phi_i/h, then
 * zeros.  Loss: mean squared error over the batch and the 3 outputs.  Optimiser:
 * Adam, beta1 = 0.9, beta2 = 0.999, eps = 1e-8, bias-corrected. */
#define SPH_MLP_NPARAM 49923
/* features of the particles in pos (float64 [3][n]); geometry and body from prm */
int sph_mlp_features(sph_ctx* ctx, const sph_relax_params* prm, const double* pos,
                     float* feats, void* stream);
/* out [n][3] = network(feats [n][128]) */
int sph_mlp_forward(sph_ctx* ctx, const float* params, const float* feats, float* out,
                    int64_t n, void* stream);
/* The same forward, fused in one launch on the fifth-generation tensor cores
 * (tcgen05.mma, bfloat16 operands in shared memory, float32 accumulation in tensor
 * memory): the activations stay on chip, global memory sees feats (float32
 * [n][128], 16-byte aligned) once and out [n][3].  Numerically the same network
 * as sph_mlp_forward (bfloat16 operands, float32 accumulation, GELU in float32);
 * the two differ by rounding order only.  A bounded wait that expires sets the
 * timeout flag, reported by sph_take_status. */
int sph_mlp_forward_tc(sph_ctx* ctx, const float* params, const float* feats, float* out,
                       int64_t n, void* stream);
/* Reads and clears the context's device timeout flag: SPH_ERR_TIMEOUT when a bounded
 * wait of a kernel expired since the last read (the results of that launch are not
 * valid), else SPH_OK.  Synchronises the stream. */
int sph_take_status(sph_ctx* ctx, void* stream);
/* gradient (float32 [SPH_MLP_NPARAM]) of the loss over a batch of b rows against
 * target [b][3]; *loss_host (nullable; if set the call synchronises) gets the loss */
int sph_mlp_grad(sph_ctx* ctx, const float* params, const float* feats, const float* target,
                 int64_t b, float* grad, double* loss_host, void* stream);
/* one Adam step (step counts from 1) on params with moments adam_m, adam_v */
int sph_mlp_train_step(sph_ctx* ctx, float* params, float* adam_m, float* adam_v,
                       int64_t step, double lr, const float* feats, const float* target,
                       int64_t b, double* loss_host, void* stream);
/* proposal move: features at pos, forward (the fused tensor-core form of
 * sph_mlp_forward_tc), pos += h * out, then particles with phi > -dp/2 are moved
 * along grad phi to phi = -dp/2 */
int sph_relax_propose(sph_ctx* ctx, const sph_relax_params* prm, const float* params,
                      double* pos, void* stream);

/* ---- a12 driven from the library: training data, training and the learned run ----
 * Plain relaxation trajectory samples for training the proposal: from pos (advanced in
 * place by snapshots * every plain steps of sph_relax_step), for k < snapshots,
 *   feats   [k n + i][128] = sph_mlp_features at x^(k every),
 *   targets [k n + i][3]   = (x_i^((k+1) every) - x_i^(k every)) / h   (float32).
 * dim 3.  The caller allocates feats [snapshots n][128] and targets [snapshots n][3]. */
int sph_relax_samples(sph_ctx* ctx, const sph_relax_params* prm, double* pos, const double* vol,
                      int snapshots, int every, float* feats, float* targets, void* stream);
/* nsteps Adam steps (sph_mlp_train_step; step numbers first_step .. first_step + nsteps - 1)
 * on minibatches of `batch` rows drawn with replacement from the `rows` samples
 * (feats [rows][128], targets [rows][3]): row b of step t is sample
 * floor(z * rows / 2^64), z = SplitMix64(SplitMix64(seed ^ SplitMix64(t)) + b), SplitMix64
 * being the generator of Steele, Lea and Flood (OOPSLA 2014) with the mixing function of its
 * public reference implementation.  The draw and the gather run
 * on the device.  *loss_host (nullable; if set the call synchronises) receives the last
 * step's minibatch loss. */
int sph_mlp_train(sph_ctx* ctx, float* params, float* adam_m, float* adam_v, int64_t first_step,
                  double lr, const float* feats, const float* targets, int64_t rows, int64_t batch,
                  int nsteps, uint64_t seed, double* loss_host, void* stream);
/* Relaxation to a residual target with an optional learned proposal.  The residual is
 * out[0] of sph_relax_residual (Laguerre-Gauss, interior particles).  With a proposal
 * (applications > 0): up to `applications` times, while the target is not met, the
 * proposal moves the particles (sph_relax_propose) and is kept only if it lowers the
 * residual (else it is undone and no further proposal is tried), then up to
 * plain_between plain steps follow; plain steps (sph_relax_step, checked every
 * check_every steps) then finish the run, until the target or max_steps plain steps.  If
 * the target is still missed, plain relaxation is the fallback: pos is reset to its
 * value at the call and relaxed plainly (up to max_steps), and that is the result.
 * Without a proposal (applications = 0) it is the plain run alone.  judge selects the
 * residual that decides: SPH_FP64 (sph_relax_residual) or SPH_FP32_KAHAN
 * (sph_relax_residual_fp32, the float32 pair sums with a float64 reduction); the
 * result's residual[] is always sph_relax_residual's.  Synchronises the stream (every
 * residual check). */
typedef struct {
    const float* proposal;          /* MLP parameters, float32 [SPH_MLP_NPARAM] on the device; may be NULL
                                       when applications = 0 */
    double target;                  /* Laguerre-Gauss residual to reach */
    int32_t max_steps;              /* cap on plain steps (of each run: learned, and fallback) */
    int32_t check_every;            /* plain steps between residual checks, >= 1 */
    int32_t applications;           /* proposal applications, >= 0 */
    int32_t plain_between;          /* plain steps after each kept proposal, >= 0 */
    int32_t judge;                  /* SPH_FP64 or SPH_FP32_KAHAN: the residual that decides */
    int32_t reserved;
} sph_relax_run_params;
typedef struct {
    int32_t steps;                  /* plain steps of the run whose result is returned */
    int32_t proposals_kept;         /* proposals that lowered the residual */
    int32_t proposals_rejected;     /* proposals undone */
    int32_t reached;                /* 1 when the final residual is <= target */
    int32_t fell_back;              /* 1 when the result is the plain fallback run */
    int32_t steps_before_fallback;  /* plain steps of the abandoned learned run */
    double residual[3];             /* final sph_relax_residual output (float64) */
    double judged;                  /* the final residual as the judge evaluated it */
} sph_relax_run_result;
int sph_relax_run(sph_ctx* ctx, const sph_relax_params* prm, double* pos, const double* vol,
                  const sph_relax_run_params* rp, sph_relax_run_result* result_host, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* SPH_H */
