"""Python binding of libsph: argument marshalling over the C ABI of include/sph.h.

PyTorch provides device memory and the current CUDA stream; every step of the
SPH path runs in libsph's kernels.  Names follow the C entry points.
"""
import ctypes

import torch

from . import _lib as L
from ._lib import (SPH_FP32_KAHAN, SPH_FP64, SPH_FUSED, SPH_LAGUERRE_GAUSS,  # noqa: F401
                   SPH_NEO_HOOKEAN, SPH_SVK, SPH_TWO_PASS, SPH_WENDLAND_C2, SPH_PASS_BATCHED,
                   SPH_PASS_COMPRESSIBLE, SPH_PASS_EULERIAN, SPH_PASS_RELAX, SPH_PASS_TLSPH, SPH_TIMER_NEIGHBORS,
                   SPH_TIMER_RELAX_ACCEL, SPH_TIMER_RELAX_UPDATE, SPH_PIPE_STREAM, SPH_PIPE_PERSISTENT,
                   SPH_PIPE_BULK, SPH_PIPE_GEOM, SPH_RING_AUTO, SPH_RING_CHUNK, SPH_RING_THREAD)

NSYM = {2: 3, 3: 6}


def _p(t):
    """Raw pointer of a tensor argument.  The C ABI reads arrays in row-major order
    ([dim][n] and the like), so a tensor with other strides is refused rather than
    passed (torch.tensor of a Fortran-ordered array, a transposed view)."""
    if t is None:
        return None
    if not t.is_contiguous():
        raise ValueError("libsph array arguments must be contiguous (got strides %s)" % (t.stride(),))
    return ctypes.c_void_p(t.data_ptr())


def _ptr(x):
    """Pointer of a device tensor (contiguous) or of a mapped HostArray buffer."""
    if isinstance(x, HostArray):
        return ctypes.c_void_p(x.dev)
    return _p(x)


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _dev_f64(x, device):
    return torch.as_tensor(x, dtype=torch.float64, device=device).contiguous()


def make_domain(dom, n):
    """sph_domain from the plain-dict description used by ``inputs``."""
    d = L.SphDomain()
    d.dim = dom["dim"]
    d.periodic_mask = sum((1 << k) for k, p in enumerate(dom["periodic"][: dom["dim"]]) if p)
    d.n = int(n)
    d.h = dom["h"]
    d.kappa = dom["kappa"]
    for k in range(3):
        d.lo[k] = dom["lo"][k] if k < dom["dim"] else 0.0
        d.len[k] = dom["len"][k] if k < dom["dim"] else 1.0
    return d


class Context:
    """Owns an sph_ctx (scratch arena and launch settings) on one CUDA device."""

    def __init__(self, device=0):
        self.lib = L.load()
        self.device = torch.device("cuda", device)
        h = ctypes.c_void_p()
        L.check("sph_create", self.lib.sph_create(ctypes.byref(h), device))
        self.h = h

    def close(self):
        if self.h:
            self.lib.sph_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_tile_pipeline(self, mode):
        """How the planned TL passes get their pair entries: SPH_PIPE_GEOM (default), _STREAM,
        _PERSISTENT or _BULK."""
        L.check("sph_set_tile_pipeline", self.lib.sph_set_tile_pipeline(self.h, int(mode)), self.h)

    def set_wait_test(self, polls):
        """Failure-detection test: polls > 0 makes the bounded waits of the bulk-copy
        deformation pass run out (no copy issued); 0 restores normal operation."""
        L.check("sph_set_wait_test", self.lib.sph_set_wait_test(self.h, int(polls)), self.h)

    def set_stage_cap(self, cap):
        L.check("sph_set_stage_cap", self.lib.sph_set_stage_cap(self.h, int(cap)), self.h)

    def set_entry_ring(self, mode):
        """How the planned Eulerian passes read their pair entries: SPH_RING_AUTO (default),
        SPH_RING_THREAD or SPH_RING_CHUNK (results do not depend on it)."""
        L.check("sph_set_entry_ring", self.lib.sph_set_entry_ring(self.h, int(mode)), self.h)

    def set_l2_persist(self, on):
        """Mark the records the planned TL passes gather persisting in L2 (default on); off
        gives the context's L2 set-aside back (synchronises the device)."""
        L.check("sph_set_l2_persist", self.lib.sph_set_l2_persist(self.h, 1 if on else 0), self.h)

    def set_relax_skin(self, skin_over_h):
        """Skin of the float32 relaxation list in units of h (0: a cell sweep every step)."""
        L.check("sph_set_relax_skin", self.lib.sph_set_relax_skin(self.h, float(skin_over_h)), self.h)

    def set_lanes(self, which, lanes):
        L.check("sph_set_lanes", self.lib.sph_set_lanes(self.h, which, lanes), self.h)

    def get_lanes(self, which):
        return self.lib.sph_get_lanes(self.h, which)

    def timing(self, on, every=1):
        """Start (clearing the counters; events around every `every`-th launch of each
        slot) or stop per-kernel event timing."""
        L.check("sph_timing_enable", self.lib.sph_timing_enable(self.h, int(every) if on else 0), self.h)

    def launches(self, slot):
        """All launches of one SPH_TIMER_* slot since timing was enabled, timed or not."""
        cnt = ctypes.c_int64()
        L.check("sph_timing_launches", self.lib.sph_timing_launches(self.h, slot, ctypes.byref(cnt)), self.h)
        return cnt.value

    def timer(self, slot):
        """(total device milliseconds, launches) recorded for one SPH_TIMER_* slot."""
        ms = ctypes.c_double()
        cnt = ctypes.c_int64()
        L.check("sph_timing_read", self.lib.sph_timing_read(self.h, slot, ctypes.byref(ms), ctypes.byref(cnt)),
                self.h)
        return ms.value, cnt.value


class HostArray:
    """Page-locked host memory mapped into the device address space (sph_host_alloc).

    ``t`` is a CPU tensor over the buffer; ``dev`` is the pointer device code uses,
    which any array field of a state struct may hold: the kernels then read and write
    the host buffer in place over the host link, with no separate copy."""

    def __init__(self, shape, dtype=torch.float64):
        import numpy as np
        self._lib = L.load()
        self.dtype = dtype
        self.shape = tuple(int(x) for x in shape)
        count = 1
        for x in self.shape:
            count *= x
        npdt = {torch.float64: np.float64, torch.float32: np.float32}[dtype]
        nbytes = count * np.dtype(npdt).itemsize
        h, d = ctypes.c_void_p(), ctypes.c_void_p()
        L.check("sph_host_alloc", self._lib.sph_host_alloc(nbytes, ctypes.byref(h), ctypes.byref(d)))
        self._host = h.value
        self.dev = d.value
        buf = (ctypes.c_char * nbytes).from_address(self._host)
        self.t = torch.from_numpy(np.frombuffer(buf, dtype=npdt).reshape(self.shape))

    def close(self):
        if self._host:
            self.t = None
            L.check("sph_host_free", self._lib.sph_host_free(self._host))
            self._host = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def kernel_eval(kernel, dim, h, kappa, precision, r):
    lib = L.load()
    r = r.contiguous()
    w = torch.empty_like(r)
    dw = torch.empty_like(r)
    L.check("sph_kernel_eval", lib.sph_kernel_eval(kernel, dim, h, kappa, precision, _p(r), _p(w), _p(dw),
                                                     r.numel(), _stream()))
    return w, dw


def cell_order(ctx, dom, pos):
    n = pos.shape[1]
    d = make_domain(dom, n)
    order = torch.empty(n, dtype=torch.int64, device=pos.device)
    L.check("sph_cell_order", ctx.lib.sph_cell_order(ctx.h, ctypes.byref(d), _p(pos), _p(order), _stream()), ctx.h)
    return order


def build_neighbors(ctx, dom, pos, cap=None):
    """CSR (row_ptr int64 [n+1], col int32 [nnz]) of the compact-support neighbour sets."""
    n = pos.shape[1]
    d = make_domain(dom, n)
    row_ptr = torch.empty(n + 1, dtype=torch.int64, device=pos.device)
    if cap is None:
        cap = max(16, n * (24 if dom["dim"] == 2 else 96))
    for _ in range(2):
        col = torch.empty(max(cap, 1), dtype=torch.int32, device=pos.device)
        nnz = ctypes.c_int64(0)
        st = ctx.lib.sph_build_neighbors(ctx.h, ctypes.byref(d), _p(pos), _p(row_ptr), _p(col), cap,
                                         ctypes.byref(nnz), _stream())
        if st == L.SPH_ERR_CAPACITY:
            cap = nnz.value
            continue
        L.check("sph_build_neighbors", st, ctx.h)
        return row_ptr, col[: nnz.value]
    raise RuntimeError("sph_build_neighbors: capacity retry failed")


def field_approx(ctx, dom, pos, vol, row_ptr, col, f, B=None, kernel=SPH_WENDLAND_C2):
    """(kernel summation [n], weak-form gradient [dim][n]) of the field f (sph_field_approx)."""
    n = pos.shape[1]
    d = make_domain(dom, n)
    s = torch.empty(n, dtype=torch.float64, device=pos.device)
    g = torch.empty((dom["dim"], n), dtype=torch.float64, device=pos.device)
    L.check("sph_field_approx", ctx.lib.sph_field_approx(ctx.h, ctypes.byref(d), kernel, _p(pos), _p(vol),
                                                          _p(row_ptr), _p(col), _p(B), _p(f), _p(s), _p(g),
                                                          _stream()), ctx.h)
    return s, g


def kgc(ctx, dom, pos, vol, row_ptr, col, kernel=SPH_WENDLAND_C2):
    n = pos.shape[1]
    d = make_domain(dom, n)
    B = torch.empty((NSYM[dom["dim"]], n), dtype=torch.float64, device=pos.device)
    fb = torch.empty(n, dtype=torch.uint8, device=pos.device)
    nfb = ctypes.c_int64(0)
    L.check("sph_kgc", ctx.lib.sph_kgc(ctx.h, ctypes.byref(d), kernel, _p(pos), _p(vol), _p(row_ptr), _p(col),
                                        _p(B), _p(fb), ctypes.byref(nfb), _stream()), ctx.h)
    return B, fb, nfb.value


def density_from_pressure(ctx, dom, c0, p):
    """drho = p / c0^2 on the device (the EOS of Sec. 3.1.1 inverted,
    sph_eulerian_density_from_pressure), for initial conditions given as pressure."""
    p = _dev_f64(p, ctx.device).contiguous()
    n = p.numel()
    prm = L.EulerianParams()
    prm.dom = make_domain(dom, n)
    prm.c0 = c0
    drho = torch.empty_like(p)
    L.check("sph_eulerian_density_from_pressure",
            ctx.lib.sph_eulerian_density_from_pressure(ctx.h, ctypes.byref(prm), _p(p), _p(drho), _stream()), ctx.h)
    return drho


class Eulerian:
    """Eulerian WCSPH state on the device (float64 arrays and, for float32 steps, packed records)."""

    def __init__(self, ctx, dom, pos, vol, B, row_ptr, col, drho, v, dt, rho0, c0, mu, eta=15.0,
                 precision=SPH_FP64, integrator=SPH_TWO_PASS, tiles=True):
        self.ctx = ctx
        dev = ctx.device
        self.n = pos.shape[1]
        self.dim = dom["dim"]
        self.prm = L.EulerianParams()
        self.prm.dom = make_domain(dom, self.n)
        self.prm.dt, self.prm.rho0, self.prm.c0, self.prm.mu, self.prm.eta = dt, rho0, c0, mu, eta
        self.prm.precision = precision
        self.prm.integrator = integrator
        self.pos = _dev_f64(pos, dev)
        self.vol = _dev_f64(vol, dev)
        self.B = _dev_f64(B, dev)
        self.row_ptr = row_ptr
        self.col = col
        self.drho = _dev_f64(drho, dev).clone()
        self.v = _dev_f64(v, dev).clone()
        self.drho_tmp = torch.empty_like(self.drho)
        self.v_tmp = torch.empty_like(self.v)
        self.rec = torch.zeros(self.n * 16, dtype=torch.float32, device=dev)
        self.rec_tmp = torch.zeros(self.n * 16, dtype=torch.float32, device=dev)
        self.st = L.EulerianState()
        for name in ("row_ptr", "col", "pos", "vol", "B", "drho", "v", "drho_tmp", "v_tmp", "rec", "rec_tmp"):
            setattr(self.st, name, getattr(self, name).data_ptr())
        self.plan = None
        if tiles and precision == SPH_FP32_KAHAN:
            # tile plan: fixed pair geometry precomputed, neighbours staged per tile (sph_eulerian_plan)
            nb = ctypes.c_int64()
            self._call("sph_eulerian_plan_bytes", ctypes.byref(nb), _stream())
            self.plan = torch.empty(max(nb.value, 16), dtype=torch.uint8, device=dev)
            self.st.plan = self.plan.data_ptr()
            self.st.plan_bytes = self.plan.numel()
        if precision == SPH_FP32_KAHAN:
            self.pack()
            if self.plan is not None:
                self._call("sph_eulerian_plan", _stream())

    def _call(self, name, *args):
        fn = getattr(self.ctx.lib, name)
        L.check(name, fn(self.ctx.h, ctypes.byref(self.prm), ctypes.byref(self.st), *args), self.ctx.h)

    def pack(self):
        self._call("sph_eulerian_pack", _stream())

    def unpack(self):
        self._call("sph_eulerian_unpack", _stream())

    def step(self, nsteps=1):
        self._call("sph_eulerian_step", int(nsteps), _stream())

    def autotune(self, trial_steps=10):
        """Pick the fastest lanes-per-particle for the float32 passes (state restored)."""
        lanes, ms = ctypes.c_int(), ctypes.c_double()
        self._call("sph_autotune_eulerian", int(trial_steps), ctypes.byref(lanes), ctypes.byref(ms), _stream())
        return lanes.value, ms.value

    def rates(self):
        drho_dt = torch.empty(self.n, dtype=torch.float64, device=self.ctx.device)
        dmom_dt = torch.empty((self.dim, self.n), dtype=torch.float64, device=self.ctx.device)
        self._call("sph_eulerian_rates", _p(drho_dt), _p(dmom_dt), _stream())
        return drho_dt, dmom_dt

    def fields(self):
        """(drho, v) as float64 device tensors (unpacked for float32 runs)."""
        if self.prm.precision == SPH_FP32_KAHAN:
            self.unpack()
        return self.drho, self.v


class Compressible:
    """Compressible Eulerian SPH state on the device (sph_compressible_*, float64):
    rho [n], mom = rho v [dim][n] and E [n] advanced in place."""

    def __init__(self, ctx, dom, pos, vol, B, row_ptr, col, rho, mom, E, dt, gamma=1.4, eta=1.0,
                 precision=SPH_FP64):
        dev = ctx.device
        self.ctx = ctx
        self.n = pos.shape[1]
        self.dim = dom["dim"]
        self.prm = L.CompressibleParams()
        self.prm.dom = make_domain(dom, self.n)
        self.prm.dt, self.prm.gamma, self.prm.eta = dt, gamma, eta
        self.prm.precision = precision
        self.pos, self.vol, self.B = _dev_f64(pos, dev), _dev_f64(vol, dev), _dev_f64(B, dev)
        self.row_ptr, self.col = row_ptr, col
        self.rho, self.mom, self.E = (_dev_f64(rho, dev).clone(), _dev_f64(mom, dev).clone(),
                                      _dev_f64(E, dev).clone())
        self.st = L.CompressibleState()
        for name in ("row_ptr", "col", "pos", "vol", "B", "rho", "mom", "E"):
            setattr(self.st, name, getattr(self, name).data_ptr())
        self.plan = None
        if precision == SPH_FP32_KAHAN:
            nb = ctypes.c_int64(0)
            self._call("sph_compressible_plan_bytes", ctypes.byref(nb), _stream())
            self.plan = torch.empty(max(nb.value, 16), dtype=torch.uint8, device=dev)
            self.st.plan, self.st.plan_bytes = self.plan.data_ptr(), self.plan.numel()
            self._call("sph_compressible_plan", _stream())

    def _call(self, name, *args):
        fn = getattr(self.ctx.lib, name)
        L.check(name, fn(self.ctx.h, ctypes.byref(self.prm), ctypes.byref(self.st), *args), self.ctx.h)

    def rates(self):
        dev = self.rho.device
        drho = torch.empty(self.n, dtype=torch.float64, device=dev)
        dmom = torch.empty((self.dim, self.n), dtype=torch.float64, device=dev)
        dE = torch.empty(self.n, dtype=torch.float64, device=dev)
        self._call("sph_compressible_rates", _p(drho), _p(dmom), _p(dE), _stream())
        return drho, dmom, dE

    def step(self, nsteps=1):
        self._call("sph_compressible_step", int(nsteps), _stream())


class TLSolid:
    """Total-Lagrangian solid state on the device."""

    def __init__(self, ctx, dom, r0, V0, B0, fixed, row_ptr, col, v, dt, rho0, lam, G, law=SPH_NEO_HOOKEAN,
                 precision=SPH_FP64, x=None, H=None, tiles=True):
        self.ctx = ctx
        dev = ctx.device
        self.n = r0.shape[1]
        self.dim = dom["dim"]
        d = self.dim
        self.prm = L.TLParams()
        self.prm.dom = make_domain(dom, self.n)
        self.prm.dt, self.prm.rho0, self.prm.lam, self.prm.G = dt, rho0, lam, G
        self.prm.law = law
        self.prm.precision = precision
        self.r0 = _dev_f64(r0, dev)
        self.V0 = _dev_f64(V0, dev)
        self.B0 = _dev_f64(B0, dev)
        self.fixed = torch.as_tensor(fixed, dtype=torch.uint8, device=dev).contiguous()
        self.row_ptr, self.col = row_ptr, col
        self.x = (self.r0.clone() if x is None else _dev_f64(x, dev).clone())
        self.v = _dev_f64(v, dev).clone()
        self.H = (torch.zeros((d * d, self.n), dtype=torch.float64, device=dev) if H is None
                  else _dev_f64(H, dev).clone())
        self.M = torch.zeros((d * d, self.n), dtype=torch.float64, device=dev)
        self.rd = torch.zeros(self.n * 8, dtype=torch.float32, device=dev)
        self.rm = torch.zeros(self.n * (16 if d == 3 else 8), dtype=torch.float32, device=dev)
        self.H32 = torch.zeros(d * d * self.n, dtype=torch.float32, device=dev)
        self.u32 = torch.zeros(d * self.n, dtype=torch.float32, device=dev)
        self.B32 = torch.zeros(NSYM[d] * self.n, dtype=torch.float32, device=dev)
        self.st = L.TLState()
        for name in ("row_ptr", "col", "r0", "V0", "B0", "fixed", "x", "v", "H", "M", "rd", "rm", "H32", "u32",
                     "B32"):
            setattr(self.st, name, getattr(self, name).data_ptr())
        self.plan = None
        if tiles and precision == SPH_FP32_KAHAN:
            # tile plan: pair factors precomputed and neighbours staged per tile (sph_tlsph_plan)
            nb = ctypes.c_int64()
            self._call("sph_tlsph_plan_bytes", ctypes.byref(nb), _stream())
            self.plan = torch.empty(max(nb.value, 16), dtype=torch.uint8, device=dev)
            self.st.plan = self.plan.data_ptr()
            self.st.plan_bytes = self.plan.numel()
        if precision == SPH_FP32_KAHAN:
            self.pack()
            if self.plan is not None:
                self._call("sph_tlsph_plan", _stream())

    def _call(self, name, *args):
        fn = getattr(self.ctx.lib, name)
        L.check(name, fn(self.ctx.h, ctypes.byref(self.prm), ctypes.byref(self.st), *args), self.ctx.h)

    def pack(self):
        self._call("sph_tlsph_pack", _stream())

    def unpack(self):
        self._call("sph_tlsph_unpack", _stream())

    def _check32(self, u, v, H):
        # the C side reads raw float32 arrays: refuse anything else before passing pointers
        d, n = self.dim, self.n
        for name, a, shape in (("u", u, (d, n)), ("v", v, (d, n)), ("H", H, (d * d, n))):
            if isinstance(a, HostArray):
                ok = a.dtype == torch.float32 and a.shape == shape
            else:
                ok = (isinstance(a, torch.Tensor) and a.is_cuda and a.dtype == torch.float32
                      and tuple(a.shape) == shape and a.is_contiguous())
            if not ok:
                raise ValueError("%s must be a contiguous float32 CUDA tensor or HostArray of shape %s" % (name, shape))

    def load32(self, u, v, H):
        """Replace the float32 form's state with u = x - r0, v, H = F - I (float32 device
        tensors or mapped HostArray buffers of shapes [dim][n], [dim][n], [dim*dim][n])."""
        self._check32(u, v, H)
        self._call("sph_tlsph_load32", _ptr(u), _ptr(v), _ptr(H), _stream())

    def store32(self, u, v, H):
        """Copy the float32 form's state (u = x - r0, v, H = F - I) out, as load32 takes it."""
        self._check32(u, v, H)
        self._call("sph_tlsph_store32", _ptr(u), _ptr(v), _ptr(H), _stream())

    def step_host32(self, u, v, H, nsteps=1):
        """nsteps float32 steps with the state kept in u, v, H (as load32 takes them): each
        step reads it in and writes it back, the copies overlapped with the passes."""
        self._check32(u, v, H)
        self._call("sph_tlsph_step_host32", _ptr(u), _ptr(v), _ptr(H), int(nsteps), _stream())

    def step(self, nsteps=1):
        self._call("sph_tlsph_step", int(nsteps), _stream())

    def autotune(self, trial_steps=10):
        """Pick the fastest lanes-per-particle for the float32 passes (state restored)."""
        lanes, ms = ctypes.c_int(), ctypes.c_double()
        self._call("sph_autotune_tlsph", int(trial_steps), ctypes.byref(lanes), ctypes.byref(ms), _stream())
        return lanes.value, ms.value

    def energy(self):
        """(kinetic, stored) energy of the float64 state in float64 (sph_tlsph_energy);
        unpacks first after float32 steps."""
        if self.prm.precision == SPH_FP32_KAHAN:
            self.unpack()
        out = (ctypes.c_double * 2)()
        self._call("sph_tlsph_energy", out, _stream())
        return out[0], out[1]

    def rates(self):
        d = self.dim
        dvdt = torch.empty((d, self.n), dtype=torch.float64, device=self.ctx.device)
        dFdt = torch.empty((d * d, self.n), dtype=torch.float64, device=self.ctx.device)
        self._call("sph_tlsph_rates", _p(dvdt), _p(dFdt), _stream())
        return dvdt, dFdt

    def fields(self):
        """(x, v, H = F - I) as float64 device tensors."""
        if self.prm.precision == SPH_FP32_KAHAN:
            self.unpack()
        return self.x, self.v, self.H


def relax_params(dom, spheres, dp, precision=SPH_FP32_KAHAN, p0=1.0, rho=1.0, n=0, kernel=SPH_LAGUERRE_GAUSS):
    """Relaxation parameters; spheres rows (cx, cy, cz, r), or circles (cx, cy, r) in 2D."""
    prm = L.RelaxParams()
    prm.dom = make_domain(dom, n)
    prm.dp, prm.p0, prm.rho = dp, p0, rho
    prm.kernel = kernel
    prm.precision = precision
    prm.n_spheres = len(spheres)
    for k, s in enumerate(spheres):
        row = [s[0], s[1], 0.0, s[2]] if len(s) == 3 else list(s[:4])
        for c in range(4):
            prm.spheres[4 * k + c] = float(row[c])
    return prm


def relax_step(ctx, prm, pos, vol, nsteps=1):
    """Advance ``nsteps`` relaxation steps of pos (float64 [dim][n] device tensor, in place)."""
    prm.dom.n = pos.shape[1]
    L.check("sph_relax_step", ctx.lib.sph_relax_step(ctx.h, ctypes.byref(prm), _p(pos), _p(vol), int(nsteps),
                                                      _stream()), ctx.h)
    return pos


def relax_accel(ctx, prm, pos, vol):
    prm.dom.n = pos.shape[1]
    acc = torch.empty_like(pos)
    L.check("sph_relax_accel", ctx.lib.sph_relax_accel(ctx.h, ctypes.byref(prm), _p(pos), _p(vol), _p(acc),
                                                        _stream()), ctx.h)
    return acc


def relax_residual(ctx, prm, pos, vol):
    prm.dom.n = pos.shape[1]
    out = (ctypes.c_double * 3)()
    L.check("sph_relax_residual", ctx.lib.sph_relax_residual(ctx.h, ctypes.byref(prm), _p(pos), _p(vol), out,
                                                              _stream()), ctx.h)
    return out[0], out[1], int(out[2])


# --------------------------------------------------------------------------- learned proposal
MLP_NPARAM = L.SPH_MLP_NPARAM


def mlp_features(ctx, prm, pos):
    prm.dom.n = pos.shape[1]
    feats = torch.empty((pos.shape[1], 128), dtype=torch.float32, device=pos.device)
    L.check("sph_mlp_features", ctx.lib.sph_mlp_features(ctx.h, ctypes.byref(prm), _p(pos), _p(feats), _stream()),
            ctx.h)
    return feats


def mlp_forward(ctx, params, feats):
    out = torch.empty((feats.shape[0], 3), dtype=torch.float32, device=feats.device)
    L.check("sph_mlp_forward", ctx.lib.sph_mlp_forward(ctx.h, _p(params), _p(feats), _p(out), feats.shape[0],
                                                        _stream()), ctx.h)
    return out


def mlp_forward_tc(ctx, params, feats, check=True):
    """The fused forward on tcgen05 tensor cores (one launch); check=True reads back the
    device status (a bounded wait that expired raises)."""
    out = torch.empty((feats.shape[0], 3), dtype=torch.float32, device=feats.device)
    L.check("sph_mlp_forward_tc", ctx.lib.sph_mlp_forward_tc(ctx.h, _p(params), _p(feats), _p(out), feats.shape[0],
                                                              _stream()), ctx.h)
    if check:
        L.check("sph_take_status", ctx.lib.sph_take_status(ctx.h, _stream()), ctx.h)
    return out


def mlp_grad(ctx, params, feats, target, with_loss=True):
    grad = torch.empty(MLP_NPARAM, dtype=torch.float32, device=feats.device)
    loss = ctypes.c_double(float("nan"))
    L.check("sph_mlp_grad", ctx.lib.sph_mlp_grad(ctx.h, _p(params), _p(feats), _p(target), feats.shape[0], _p(grad),
                                                  ctypes.byref(loss) if with_loss else None, _stream()), ctx.h)
    return grad, loss.value


class MLPTrainer:
    """float32 master parameters and Adam moments on the device."""

    def __init__(self, ctx, params, lr=1e-3):
        self.ctx = ctx
        self.params = torch.as_tensor(params, dtype=torch.float32, device=ctx.device).contiguous().clone()
        self.m = torch.zeros_like(self.params)
        self.v = torch.zeros_like(self.params)
        self.step_count = 0
        self.lr = lr

    def train(self, feats, targets, nsteps, batch=4096, seed=0, with_loss=True):
        """nsteps Adam steps on minibatches drawn on the device from (feats, targets)
        (sph_mlp_train); returns the last step's loss (nan without with_loss)."""
        loss = ctypes.c_double(float("nan"))
        L.check("sph_mlp_train", self.ctx.lib.sph_mlp_train(
            self.ctx.h, _p(self.params), _p(self.m), _p(self.v), self.step_count + 1, float(self.lr), _p(feats),
            _p(targets), feats.shape[0], int(batch), int(nsteps), int(seed) & 0xFFFFFFFFFFFFFFFF,
            ctypes.byref(loss) if with_loss else None, _stream()), self.ctx.h)
        self.step_count += int(nsteps)
        return loss.value

    def step(self, feats, target, with_loss=False):
        self.step_count += 1
        loss = ctypes.c_double(float("nan"))
        L.check("sph_mlp_train_step", self.ctx.lib.sph_mlp_train_step(
            self.ctx.h, _p(self.params), _p(self.m), _p(self.v), self.step_count, float(self.lr), _p(feats),
            _p(target), feats.shape[0], ctypes.byref(loss) if with_loss else None, _stream()), self.ctx.h)
        return loss.value


def relax_samples(ctx, prm, pos, vol, snapshots, every):
    """Plain-trajectory training samples (sph_relax_samples): features [snapshots n, 128]
    and targets (x^{t+every} - x^t)/h [snapshots n, 3], float32; pos is advanced in place."""
    n = pos.shape[1]
    prm.dom.n = n
    feats = torch.empty((snapshots * n, 128), dtype=torch.float32, device=pos.device)
    targets = torch.empty((snapshots * n, 3), dtype=torch.float32, device=pos.device)
    L.check("sph_relax_samples", ctx.lib.sph_relax_samples(ctx.h, ctypes.byref(prm), _p(pos), _p(vol),
                                                            int(snapshots), int(every), _p(feats), _p(targets),
                                                            _stream()), ctx.h)
    return feats, targets


def relax_residual_fp32(ctx, prm, pos, vol):
    """The Laguerre-Gauss residual from float32 pair sums (sph_relax_residual_fp32):
    (residual, count)."""
    prm.dom.n = pos.shape[1]
    out = (ctypes.c_double * 3)()
    L.check("sph_relax_residual_fp32", ctx.lib.sph_relax_residual_fp32(ctx.h, ctypes.byref(prm), _p(pos), _p(vol),
                                                                        out, _stream()), ctx.h)
    return out[0], int(out[2])


def relax_run(ctx, prm, pos, vol, target, max_steps, proposal=None, applications=3, plain_between=10,
              check_every=10, judge=SPH_FP64):
    """Relaxation of pos (in place) to the residual target (sph_relax_run): with a proposal,
    judged by the residual, plain relaxation finishing the run and as the fallback.
    Returns the sph_relax_run_result fields as a dict."""
    prm.dom.n = pos.shape[1]
    rp = L.RelaxRunParams()
    rp.proposal = _p(proposal) if proposal is not None else None
    rp.target = float(target)
    rp.max_steps, rp.check_every = int(max_steps), int(check_every)
    rp.applications = int(applications) if proposal is not None else 0
    rp.plain_between = int(plain_between)
    rp.judge = int(judge)
    out = L.RelaxRunResult()
    L.check("sph_relax_run", ctx.lib.sph_relax_run(ctx.h, ctypes.byref(prm), _p(pos), _p(vol), ctypes.byref(rp),
                                                    ctypes.byref(out), _stream()), ctx.h)
    return {"steps": out.steps, "kept": out.proposals_kept, "rejected": out.proposals_rejected,
            "reached": bool(out.reached), "fell_back": bool(out.fell_back),
            "steps_before_fallback": out.steps_before_fallback, "residual": list(out.residual),
            "judged": out.judged}


def relax_propose(ctx, prm, params, pos):
    prm.dom.n = pos.shape[1]
    L.check("sph_relax_propose", ctx.lib.sph_relax_propose(ctx.h, ctypes.byref(prm), _p(params), _p(pos),
                                                            _stream()), ctx.h)
    return pos
