"""ctypes declarations of the libsph C ABI (include/sph.h).

Argument marshalling only: every computation runs in libsph's CUDA kernels.
The library is loaded on first use; a missing build raises immediately (there
is no fallback path).
"""
import ctypes
import os

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "lib", "libsph.so")
HEADER = os.path.join(os.path.dirname(PKG), "include", "sph.h")

SPH_OK, SPH_ERR_ARG, SPH_ERR_CAPACITY, SPH_ERR_CUDA, SPH_ERR_TIMEOUT, SPH_ERR_NONFINITE, SPH_ERR_LIMIT = range(7)
SPH_STATIC_MAX_PARTICLES = 1 << 20
SPH_STATIC_MAX_CELLS = 1 << 20
SPH_WENDLAND_C2, SPH_LAGUERRE_GAUSS = 0, 1
SPH_FP64, SPH_FP32_KAHAN = 0, 1
SPH_TWO_PASS, SPH_FUSED = 0, 1
SPH_SVK, SPH_NEO_HOOKEAN = 0, 1
SPH_PASS_EULERIAN, SPH_PASS_TLSPH, SPH_PASS_RELAX, SPH_PASS_BATCHED, SPH_PASS_COMPRESSIBLE = 0, 1, 2, 3, 4
SPH_PIPE_STREAM, SPH_PIPE_PERSISTENT, SPH_PIPE_BULK, SPH_PIPE_GEOM = 0, 1, 2, 3
SPH_RING_AUTO, SPH_RING_THREAD, SPH_RING_CHUNK = 0, 1, 2
SPH_TIMER_BATCH_STEP = 9
SPH_MAX_SPHERES = 16
(SPH_TIMER_TL_STRESS, SPH_TIMER_TL_MOMENTUM, SPH_TIMER_TL_DEFORM, SPH_TIMER_EU_MOMENTUM, SPH_TIMER_EU_MASS,
 SPH_TIMER_EU_FUSED, SPH_TIMER_NEIGHBORS, SPH_TIMER_RELAX_ACCEL, SPH_TIMER_RELAX_UPDATE) = range(9)

c_i32, c_i64, c_dbl, c_vp = ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_void_p


class SphDomain(ctypes.Structure):
    _fields_ = [("dim", c_i32), ("periodic_mask", ctypes.c_uint32), ("n", c_i64), ("h", c_dbl),
                ("kappa", c_dbl), ("lo", c_dbl * 3), ("len", c_dbl * 3)]


class EulerianParams(ctypes.Structure):
    _fields_ = [("dom", SphDomain), ("dt", c_dbl), ("rho0", c_dbl), ("c0", c_dbl), ("mu", c_dbl),
                ("eta", c_dbl), ("precision", c_i32), ("integrator", c_i32)]


class EulerianState(ctypes.Structure):
    _fields_ = [(name, c_vp) for name in ("row_ptr", "col", "pos", "vol", "B", "drho", "v", "drho_tmp",
                                          "v_tmp", "rec", "rec_tmp", "plan")] + [
        ("plan_bytes", c_i64), ("plan_nnz", c_i64), ("plan_maxm", c_i32), ("plan_maxrow", c_i32)]


class TLParams(ctypes.Structure):
    _fields_ = [("dom", SphDomain), ("dt", c_dbl), ("rho0", c_dbl), ("lam", c_dbl), ("G", c_dbl),
                ("law", c_i32), ("precision", c_i32)]


class TLState(ctypes.Structure):
    _fields_ = [(name, c_vp) for name in ("row_ptr", "col", "r0", "V0", "B0", "fixed", "x", "v", "H", "M",
                                          "rd", "rm", "H32", "u32", "B32", "plan")] + [
        ("plan_bytes", c_i64), ("plan_nnz", c_i64), ("plan_maxm", c_i32), ("plan_maxrow", c_i32)]


class BatchCase(ctypes.Structure):
    _fields_ = [("offset", c_i64), ("n", c_i64), ("dim", c_i32), ("periodic_mask", ctypes.c_uint32),
                ("h", c_dbl), ("dt", c_dbl), ("rho0", c_dbl), ("c0", c_dbl), ("mu", c_dbl), ("eta", c_dbl),
                ("len", c_dbl * 3), ("plan", c_vp), ("plan_nnz", c_i64), ("plan_maxm", c_i32),
                ("plan_maxrow", c_i32)]


class BatchState(ctypes.Structure):
    _fields_ = [(name, c_vp) for name in ("row_ptr", "col", "rec", "rec_tmp")]


class RelaxParams(ctypes.Structure):
    _fields_ = [("dom", SphDomain), ("dp", c_dbl), ("p0", c_dbl), ("rho", c_dbl), ("kernel", c_i32),
                ("precision", c_i32), ("n_spheres", c_i32), ("reserved", c_i32),
                ("spheres", c_dbl * (4 * SPH_MAX_SPHERES))]


class RelaxRunParams(ctypes.Structure):
    _fields_ = [("proposal", c_vp), ("target", c_dbl), ("max_steps", c_i32), ("check_every", c_i32),
                ("applications", c_i32), ("plain_between", c_i32), ("judge", c_i32), ("reserved", c_i32)]


class RelaxRunResult(ctypes.Structure):
    _fields_ = [("steps", c_i32), ("proposals_kept", c_i32), ("proposals_rejected", c_i32), ("reached", c_i32),
                ("fell_back", c_i32), ("steps_before_fallback", c_i32), ("residual", c_dbl * 3), ("judged", c_dbl)]


class CompressibleParams(ctypes.Structure):
    _fields_ = [("dom", SphDomain), ("dt", c_dbl), ("gamma", c_dbl), ("eta", c_dbl), ("precision", c_i32),
                ("reserved", c_i32)]


class CompressibleState(ctypes.Structure):
    _fields_ = [(name, c_vp) for name in ("row_ptr", "col", "pos", "vol", "B", "rho", "mom", "E", "plan")] + [
        ("plan_bytes", ctypes.c_int64), ("plan_width", c_i32), ("reserved", c_i32)]


_P = ctypes.POINTER
_SIGNATURES = {
    "sph_create": (ctypes.c_int, [_P(c_vp), ctypes.c_int]),
    "sph_destroy": (ctypes.c_int, [c_vp]),
    "sph_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "sph_last_cuda_error": (ctypes.c_int, [c_vp]),
    "sph_set_lanes": (ctypes.c_int, [c_vp, ctypes.c_int, ctypes.c_int]),
    "sph_get_lanes": (ctypes.c_int, [c_vp, ctypes.c_int]),
    "sph_timing_enable": (ctypes.c_int, [c_vp, ctypes.c_int]),
    "sph_timing_read": (ctypes.c_int, [c_vp, ctypes.c_int, _P(c_dbl), _P(c_i64)]),
    "sph_timing_launches": (ctypes.c_int, [c_vp, ctypes.c_int, _P(ctypes.c_int64)]),
    "sph_kernel_eval": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, c_dbl, c_dbl, ctypes.c_int, c_vp, c_vp, c_vp,
                                       c_i64, c_vp]),
    "sph_cell_order": (ctypes.c_int, [c_vp, _P(SphDomain), c_vp, c_vp, c_vp]),
    "sph_build_neighbors": (ctypes.c_int, [c_vp, _P(SphDomain), c_vp, c_vp, c_vp, c_i64, _P(c_i64), c_vp]),
    "sph_build_neighbors_static": (ctypes.c_int, [_P(SphDomain), c_vp, c_vp, c_vp, c_i64, _P(c_i64), c_vp]),
    "sph_kgc": (ctypes.c_int, [c_vp, _P(SphDomain), ctypes.c_int, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, _P(c_i64),
                               c_vp]),
    "sph_eulerian_pack": (ctypes.c_int, [c_vp, _P(EulerianParams), _P(EulerianState), c_vp]),
    "sph_eulerian_unpack": (ctypes.c_int, [c_vp, _P(EulerianParams), _P(EulerianState), c_vp]),
    "sph_eulerian_density_from_pressure": (ctypes.c_int, [c_vp, _P(EulerianParams), c_vp, c_vp, c_vp]),
    "sph_eulerian_rates": (ctypes.c_int, [c_vp, _P(EulerianParams), _P(EulerianState), c_vp, c_vp, c_vp]),
    "sph_eulerian_step": (ctypes.c_int, [c_vp, _P(EulerianParams), _P(EulerianState), ctypes.c_int, c_vp]),
    "sph_tlsph_pack": (ctypes.c_int, [c_vp, _P(TLParams), _P(TLState), c_vp]),
    "sph_tlsph_unpack": (ctypes.c_int, [c_vp, _P(TLParams), _P(TLState), c_vp]),
    "sph_tlsph_load32": (ctypes.c_int, [c_vp, _P(TLParams), _P(TLState), c_vp, c_vp, c_vp, c_vp]),
    "sph_tlsph_store32": (ctypes.c_int, [c_vp, _P(TLParams), _P(TLState), c_vp, c_vp, c_vp, c_vp]),
    "sph_tlsph_step_host32": (ctypes.c_int, [c_vp, _P(TLParams), _P(TLState), c_vp, c_vp, c_vp, ctypes.c_int, c_vp]),
    "sph_tlsph_energy": (ctypes.c_int, [c_vp, _P(TLParams), _P(TLState), c_vp, c_vp]),
    "sph_tlsph_rates": (ctypes.c_int, [c_vp, _P(TLParams), _P(TLState), c_vp, c_vp, c_vp]),
    "sph_tlsph_step": (ctypes.c_int, [c_vp, _P(TLParams), _P(TLState), ctypes.c_int, c_vp]),
    "sph_relax_step": (ctypes.c_int, [c_vp, _P(RelaxParams), c_vp, c_vp, ctypes.c_int, c_vp]),
    "sph_relax_accel": (ctypes.c_int, [c_vp, _P(RelaxParams), c_vp, c_vp, c_vp, c_vp]),
    "sph_relax_residual": (ctypes.c_int, [c_vp, _P(RelaxParams), c_vp, c_vp, _P(c_dbl), c_vp]),
    "sph_mlp_features": (ctypes.c_int, [c_vp, _P(RelaxParams), c_vp, c_vp, c_vp]),
    "sph_mlp_forward": (ctypes.c_int, [c_vp, c_vp, c_vp, c_vp, c_i64, c_vp]),
    "sph_mlp_forward_tc": (ctypes.c_int, [c_vp, c_vp, c_vp, c_vp, c_i64, c_vp]),
    "sph_take_status": (ctypes.c_int, [c_vp, c_vp]),
    "sph_mlp_grad": (ctypes.c_int, [c_vp, c_vp, c_vp, c_vp, c_i64, c_vp, _P(c_dbl), c_vp]),
    "sph_mlp_train_step": (ctypes.c_int, [c_vp, c_vp, c_vp, c_vp, c_i64, c_dbl, c_vp, c_vp, c_i64, _P(c_dbl),
                                          c_vp]),
    "sph_relax_propose": (ctypes.c_int, [c_vp, _P(RelaxParams), c_vp, c_vp, c_vp]),
    "sph_relax_residual_fp32": (ctypes.c_int, [c_vp, _P(RelaxParams), c_vp, c_vp, c_vp, c_vp]),
    "sph_relax_samples": (ctypes.c_int, [c_vp, _P(RelaxParams), c_vp, c_vp, ctypes.c_int, ctypes.c_int, c_vp, c_vp,
                                         c_vp]),
    "sph_mlp_train": (ctypes.c_int, [c_vp, c_vp, c_vp, c_vp, c_i64, c_dbl, c_vp, c_vp, c_i64, c_i64, ctypes.c_int,
                                     ctypes.c_uint64, _P(c_dbl), c_vp]),
    "sph_relax_run": (ctypes.c_int, [c_vp, _P(RelaxParams), c_vp, c_vp, _P(RelaxRunParams), _P(RelaxRunResult),
                                     c_vp]),
    "sph_eulerian_plan_bytes": (ctypes.c_int, [c_vp, _P(EulerianParams), _P(EulerianState), _P(c_i64), c_vp]),
    "sph_eulerian_plan": (ctypes.c_int, [c_vp, _P(EulerianParams), _P(EulerianState), c_vp]),
    "sph_tlsph_plan_bytes": (ctypes.c_int, [c_vp, _P(TLParams), _P(TLState), _P(c_i64), c_vp]),
    "sph_tlsph_plan": (ctypes.c_int, [c_vp, _P(TLParams), _P(TLState), c_vp]),
    "sph_set_stage_cap": (ctypes.c_int, [c_vp, ctypes.c_int]),
    "sph_set_entry_ring": (ctypes.c_int, [c_vp, ctypes.c_int]),
    "sph_set_l2_persist": (ctypes.c_int, [c_vp, ctypes.c_int]),
    "sph_set_relax_skin": (ctypes.c_int, [c_vp, ctypes.c_double]),
    "sph_compressible_rates": (ctypes.c_int, [c_vp, _P(CompressibleParams), _P(CompressibleState), c_vp, c_vp,
                                              c_vp, c_vp]),
    "sph_compressible_step": (ctypes.c_int, [c_vp, _P(CompressibleParams), _P(CompressibleState), ctypes.c_int,
                                             c_vp]),
    "sph_compressible_plan_bytes": (ctypes.c_int, [c_vp, _P(CompressibleParams), _P(CompressibleState),
                                                   _P(ctypes.c_int64), c_vp]),
    "sph_compressible_plan": (ctypes.c_int, [c_vp, _P(CompressibleParams), _P(CompressibleState), c_vp]),
    "sph_field_approx": (ctypes.c_int, [c_vp, _P(SphDomain), ctypes.c_int, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp,
                                        c_vp, c_vp, c_vp]),
    "sph_host_alloc": (ctypes.c_int, [ctypes.c_size_t, ctypes.POINTER(c_vp), ctypes.POINTER(c_vp)]),
    "sph_host_free": (ctypes.c_int, [c_vp]),
    "sph_set_tile_pipeline": (ctypes.c_int, [c_vp, ctypes.c_int]),
    "sph_set_wait_test": (ctypes.c_int, [c_vp, ctypes.c_uint32]),
    "sph_autotune_eulerian": (ctypes.c_int, [c_vp, _P(EulerianParams), _P(EulerianState), ctypes.c_int,
                                             _P(ctypes.c_int), _P(c_dbl), c_vp]),
    "sph_autotune_tlsph": (ctypes.c_int, [c_vp, _P(TLParams), _P(TLState), ctypes.c_int, _P(ctypes.c_int),
                                          _P(c_dbl), c_vp]),
    "sph_eulerian_step_batched":(ctypes.c_int, [c_vp, c_vp, ctypes.c_int, _P(BatchState), ctypes.c_int, c_vp]),
    "sph_autotune_batched": (ctypes.c_int, [c_vp, c_vp, ctypes.c_int, _P(BatchState), ctypes.c_int,
                                            _P(ctypes.c_int), _P(ctypes.c_int), _P(c_dbl), c_vp]),
}
SPH_MLP_NPARAM = 49923

_lib = None


class SphError(RuntimeError):
    def __init__(self, name, status, cuda_error=0):
        self.status = status
        msg = "%s failed: %s" % (name, _lib.sph_status_string(status).decode() if _lib else status)
        if status == SPH_ERR_CUDA:
            msg += " (cudaError %d)" % cuda_error
        super().__init__(msg)


def load():
    """Load libsph.so (built by ``__graft_entry__.build()``); raise if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libsph.so is not built (%s); run __graft_entry__.build() first" % LIB_PATH)
    lib = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in _SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def check(name, status, ctx=None):
    if status != SPH_OK:
        err = _lib.sph_last_cuda_error(ctx) if (ctx and status == SPH_ERR_CUDA) else 0
        raise SphError(name, status, err)
