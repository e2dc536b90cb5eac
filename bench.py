"""Benchmark of the truncated-kernel SPH hot path on GB300.

Default workload: the 3D total-Lagrangian oscillating cantilever plate
(0.2 x 0.02 x 0.2 m, dp = 1 mm, 816,000 particles, neo-Hookean rho0 = 1000,
E = 2e6 Pa, nu = 0.3975, clamped 4-layer root, first-mode initial velocity of
amplitude 0.05 c0), float32 pair loops with compensated sums and float64 KGC,
truncated Wendland cut-off 1.6h.  A step is one time step: the momentum pass
(Eq. 30) and the deformation-rate pass (Eq. 31, with the fused stress update),
i.e. 2 x nnz directed pair interactions.  The same workload is also timed at the
standard 2h cut-off and in plain float64, and the float32 result is compared
with the float64 one after the same steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line.  Under torchrun (N > 1) every rank runs an independent
replica (weak scaling; the method needs no data exchange between replicas).
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "ms/step & pair-interactions/s, 1.6h vs 2h cut-off, at matched error vs FP64"
UNIT = "pair-interactions/s"
WORKLOAD = ("3D total-Lagrangian SPH oscillating cantilever plate 0.2x0.02x0.2 m, dp=0.001 m "
            "(816,000 particles), neo-Hookean rho0=1000 E=2e6 nu=0.3975, clamped 4-layer root, "
            "first-mode initial velocity 0.05*c0, truncated Wendland kernel at 1.6h, "
            "FP32 pair loops with Kahan sums, FP64 KGC")
L2_BYTES = 129 * 1024 * 1024


def _dist_info():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# --------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples of the SM clock and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 8:
                self.rows.append(parts)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=5)
        sm = [float(r[0]) for r in self.rows if _isnum(r[0])]
        mx = [float(r[1]) for r in self.rows if _isnum(r[1])]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in self.rows for k in range(4) if r[4 + k].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


TIMER_EVERY = 10      # headline: CUDA events around every 10th launch of each pass


def _isnum(s):
    try:
        float(s)
        return True
    except ValueError:
        return False


# --------------------------------------------------------------------------- setup
def _setup_plate(api, inputs, ctx, kappa, dp=0.001):
    return _setup_solid(api, ctx, inputs.plate(dp=dp, kappa=kappa))


def _setup_solid(api, ctx, c):
    """A total-Lagrangian case of inputs (plate, columns) on the device, in Morton order,
    with its lists and correction matrices."""
    import torch
    d = c["domain"]
    dev = ctx.device
    r0 = torch.tensor(c["r0"], dtype=torch.float64, device=dev)
    order = api.cell_order(ctx, d, r0)
    r0 = r0[:, order].contiguous()
    oh = order.cpu().numpy()
    vol = torch.tensor(c["vol"][oh], dtype=torch.float64, device=dev)
    rp, col = api.build_neighbors(ctx, d, r0)
    B0, fb, nfb = api.kgc(ctx, d, r0, vol, rp, col)
    # inv: the position of each input particle in this case's cell order (the order depends
    # on the cut-off, so fields of two cut-offs are compared through it)
    inv = torch.empty_like(order)
    inv[order] = torch.arange(order.numel(), device=order.device)
    return dict(c=c, d=d, r0=r0, vol=vol, rp=rp, col=col, B0=B0, v=c["v"][:, oh], fixed=c["fixed"][oh],
                nnz=int(col.numel()), n=int(r0.shape[1]), nfb=nfb, inv=inv)


def _solid(api, ctx, s, precision, tiles=True):
    c = s["c"]
    return api.TLSolid(ctx, s["d"], s["r0"], s["vol"], s["B0"], s["fixed"], s["rp"], s["col"], s["v"], c["dt"],
                       c["rho0"], c["lam"], c["G"], law=api.SPH_NEO_HOOKEAN, precision=precision, tiles=tiles)


def _time_steps(ctx, sol, steps, warmup, world, clocks=None):
    """Device time of `steps` time steps after `warmup` untimed ones (max over ranks)."""
    import torch
    sol.step(warmup)
    torch.cuda.synchronize()
    _barrier(world)
    stream = torch.cuda.current_stream()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    if clocks:
        clocks.start()
        time.sleep(0.3)
    torch.cuda.synchronize()
    ev0.record(stream)
    sol.step(steps)
    ev1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop() if clocks else None
    _barrier(world)
    ms = ev0.elapsed_time(ev1)
    return _max_over_ranks(ms, world), clk


def _barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def _reduce_over_ranks(x, world, op):
    """All-reduce of one float64 over the ranks (NCCL on the GPU, or a gloo group)."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=op)
    return float(t.item())


def _max_over_ranks(x, world):
    import torch.distributed as dist
    return _reduce_over_ranks(x, world, dist.ReduceOp.MAX) if world > 1 else x


def _sum_over_ranks(x, world):
    import torch.distributed as dist
    return _reduce_over_ranks(x, world, dist.ReduceOp.SUM) if world > 1 else x


def _alg_bytes_tl(n, nnz):
    """Algorithmic bytes of one float32 TL step, by pass: the bytes the method must move
    (state once per pass, indices, row offsets); a plan's precomputed pair entries are not
    counted (they trade arithmetic for bytes).

    momentum pass:  row_ptr 8 + own RM record 64 + own velocity read/write 32 per particle,
                    col 4 per pair;
    deformation pass: row_ptr 8 + own RD record 32 + B0 24 + H read/write 72 + u read/write 24
                      + M write 48 per particle, col 4 per pair.
    Neighbour records (RM, RD) are counted once per particle: they are re-read from L1/L2."""
    mom = n * (8 + 64 + 32) + 4 * nnz
    defo = n * (8 + 32 + 24 + 72 + 24 + 48) + 4 * nnz
    return mom, defo


def _cpu_baseline(steps_cap_s=12.0, dp=0.003):
    """The oracle's TL step on a reduced plate (dp = 3 mm), timed on the host cores: on all
    of them (the pair sums over row blocks on a spawned process pool, oracle.pool, bitwise
    the single-process step) and on one (plain numpy).  About steps_cap_s seconds each."""
    from oracle import kgc as OK
    from oracle import neighbors as ON
    from oracle import pool as OP
    from oracle import tlsph as OT
    from paper_2405_05155_gb300 import inputs
    c = inputs.plate(dp=dp, kappa=1.6)
    d = c["domain"]
    dom = ON.Domain(d["dim"], d["h"], d["kappa"], d["lo"], d["len"], d["periodic"])
    rp, col = ON.neighbors_cells(c["r0"], dom)
    B0, _ = OK.kgc(c["r0"], c["vol"], rp, col, dom)
    prm = OT.TLParams(dom, c["dt"], c["rho0"], c["lam"], c["G"], OT.NEO_HOOKEAN)
    n = c["r0"].shape[1]

    def timed(step):
        x, v, F = c["r0"].copy(), c["v"].copy(), np.tile(np.eye(3), (n, 1, 1))
        x, v, F = step(x, v, F)          # warm-up (the pool's workers start here)
        steps = 0
        t0 = time.perf_counter()
        while time.perf_counter() - t0 < steps_cap_s or steps < 3:
            x, v, F = step(x, v, F)
            steps += 1
        return steps, time.perf_counter() - t0, v

    cores = OP.host_cores()
    with OP.PoolStep(c["r0"], c["vol"], B0, c["fixed"], rp, col, prm, workers=cores) as ps:
        steps_all, el_all, v_all = timed(ps.step)
    steps_one, el_one, _ = timed(lambda x, v, F: OT.step(c["r0"], c["vol"], B0, c["fixed"], x, v, F, rp, col, prm))
    pairs = 2 * col.size
    return {"value": pairs * steps_all / el_all, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "float64 numpy oracle, plate at dp=%g m (%d particles, nnz=%d): %d time steps in %.1f s "
                      "(%.1f ms/step) on %d host cores (the two pair sums over row blocks on a spawned process "
                      "pool, bitwise the single-process step); single core: %d steps in %.1f s (%.1f ms/step)"
                      % (dp, n, col.size, steps_all, el_all, 1e3 * el_all / steps_all, cores, steps_one, el_one,
                         1e3 * el_one / steps_one),
            "ms_per_step": 1e3 * el_all / steps_all, "particles": n,
            "single_core": {"value": pairs * steps_one / el_one, "ms_per_step": 1e3 * el_one / steps_one,
                            "cores": 1}}


# --------------------------------------------------------------------------- other rows
def _event_ms(fn):
    import torch
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1)


def _roof(bytes_per_launch, ms_per_launch, peak):
    gbs = bytes_per_launch / (ms_per_launch * 1e-3) / 1e9
    return {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s", "frac": gbs / peak,
            "algorithmic_bytes_per_launch": bytes_per_launch}


def _eulerian_case(api, ctx, case, precision, tiles=True):
    import torch
    d = case["domain"]
    dev = ctx.device
    pos = torch.tensor(case["pos"], dtype=torch.float64, device=dev)
    order = api.cell_order(ctx, d, pos)
    pos = pos[:, order].contiguous()
    oh = order.cpu().numpy()
    vol = torch.tensor(case["vol"][oh], dtype=torch.float64, device=dev)
    rp, col = api.build_neighbors(ctx, d, pos)
    B, _, nfb = api.kgc(ctx, d, pos, vol, rp, col)
    drho = api.density_from_pressure(ctx, d, case["c0"], torch.tensor(case["p"], device=dev)[order])
    sim = api.Eulerian(ctx, d, pos, vol, B, rp, col, drho, case["v"][:, oh], case["dt"],
                       case["rho0"], case["c0"], case["mu"], precision=precision, tiles=tiles)
    return sim, int(col.numel()), oh


def _bench_tgv3d(api, inputs, ctx, steps, peak):
    """3D Taylor-Green, 128^3 periodic cube, Re = 1600: float32 at 1.6h and 2h, float64 at 1.6h."""
    import torch
    from paper_2405_05155_gb300._lib import SPH_TIMER_EU_MASS, SPH_TIMER_EU_MOMENTUM
    out = {"workload": "3D Eulerian WCSPH Taylor-Green vortex, periodic cube 2*pi, 128^3 = 2,097,152 particles, "
                       "Re=1600, h=1.3dp, two-pass step, FP32+Kahan (and FP64)"}
    res = {}
    vend = {}
    for kappa in (1.6, 2.0):
        case = inputs.tgv3d(n=128, kappa=kappa)
        sim, nnz, oh = _eulerian_case(api, ctx, case, api.SPH_FP32_KAHAN)
        _, v_start = sim.fields()
        ke0 = float(torch.sum(v_start * v_start))
        lanes, _ = sim.autotune(3)
        sim.step(3)
        ctx.timing(True, every=TIMER_EVERY)
        ms = _event_ms(lambda: sim.step(steps))
        tm, nm = ctx.timer(SPH_TIMER_EU_MOMENTUM)
        tc, nc = ctx.timer(SPH_TIMER_EU_MASS)
        ctx.timing(False)
        n = sim.n
        per_pass = n * (8 + 64 + 16) + 4 * nnz       # row_ptr, own 64-byte record, (v, drho) write, col
        dom_ms = max(tm / max(nm, 1), tc / max(nc, 1))
        r = {"ms_per_step": ms / steps, "pair_interactions_per_s": 2 * nnz * steps / (ms * 1e-3), "nnz": nnz,
             "lanes": lanes, "pass_ms": {"momentum": tm / max(nm, 1), "continuity": tc / max(nc, 1)},
             "roofline": _roof(per_pass, dom_ms, peak)}
        _, v_end = sim.fields()
        inv = torch.empty(len(oh), dtype=torch.int64, device=v_end.device)
        inv[torch.as_tensor(oh, device=v_end.device)] = torch.arange(len(oh), device=v_end.device)
        vend[kappa] = v_end[:, inv].clone()       # input order: each cut-off has its own cell order
        # kinetic-energy decay rate over the run against the initial viscous rate 6 nu of the
        # Taylor-Green field (an eigenfunction of the Laplacian with eigenvalue -3; the
        # nonlinear term conserves energy), a closed form for early times
        t_run = (3 + steps) * case["dt"]
        nu = case["mu"] / case["rho0"]
        rate = -math.log(float(torch.sum(v_end * v_end)) / ke0) / t_run
        r["ke_decay"] = {"t": t_run, "rate_fit": rate, "rate_viscous_6nu": 6.0 * nu, "ratio": rate / (6.0 * nu)}
        if kappa == 1.6:
            d32, v32 = [t.clone() for t in sim.fields()]
            sim64, _, _ = _eulerian_case(api, ctx, case, api.SPH_FP64)
            sim64.step(3)
            n64 = max(5, steps // 10)
            ms64 = _event_ms(lambda: sim64.step(n64))
            r["fp64_ms_per_step"] = ms64 / n64
            # same number of steps from the same state for the error
            sim64b, _, _ = _eulerian_case(api, ctx, case, api.SPH_FP64)
            sim64b.step(3 + steps)
            d64, v64 = sim64b.fields()
            r["l2_fp32_vs_fp64"] = {"drho": float(torch.linalg.norm(d32 - d64) / torch.linalg.norm(d64)),
                                    "v": float(torch.linalg.norm(v32 - v64) / torch.linalg.norm(v64))}
            del sim64, sim64b
        res["kappa_%.1f" % kappa] = r
        del sim
    out.update(res)
    out["alpha_TW_over_SW"] = res["kappa_1.6"]["ms_per_step"] / res["kappa_2.0"]["ms_per_step"]
    out["l2_v_tw_vs_sw"] = float(torch.linalg.norm(vend[1.6] - vend[2.0]) / torch.linalg.norm(vend[2.0]))
    out["matched_accuracy_criterion"] = ("kinetic-energy decay rate of 1.6h within 10 % of 2h's, and the velocity "
                                         "fields within 1e-3 relative L2 after the same steps")
    k16, k20 = res["kappa_1.6"]["ke_decay"]["rate_fit"], res["kappa_2.0"]["ke_decay"]["rate_fit"]
    out["matched_accuracy"] = bool(abs(k16 / k20 - 1.0) <= 0.1 and out["l2_v_tw_vs_sw"] <= 1e-3)
    return out


def _bench_tgv2d(api, inputs, ctx):
    """Plain method: 2D Taylor-Green 50x50, FP64, 200 steps, TW and SW, error vs the closed form."""
    import torch
    out = {"workload": "2D Eulerian WCSPH Taylor-Green vortex, periodic unit square 50x50, Re=100, FP64, 200 steps"}
    for kappa in (1.6, 2.0):
        case = inputs.tgv2d(nx=50, kappa=kappa)
        sim, nnz, oh = _eulerian_case(api, ctx, case, api.SPH_FP64)
        ms = _event_ms(lambda: sim.step(200))
        _, v = sim.fields()
        t = 200 * case["dt"]
        exact = torch.tensor(inputs.tgv2d_exact_velocity(case["pos"][:, oh], case["U"], case["nu"], t),
                             device=ctx.device)
        out["kappa_%.1f" % kappa] = {"ms_per_step": ms / 200, "pair_interactions_per_s": 2 * nnz * 200 / (ms * 1e-3),
                                     "l2_v_vs_closed_form": float(torch.linalg.norm(v - exact) /
                                                                  torch.linalg.norm(exact))}
    out["matched_accuracy"] = (out["kappa_1.6"]["l2_v_vs_closed_form"] <= 1.1 * out["kappa_2.0"]["l2_v_vs_closed_form"])
    # the same cases run on to t = 1: the velocity amplitude A(t) = sqrt(2 <|v|^2>)/U sampled
    # every 50 steps and its decay rate fitted (least squares on log A) against the closed
    # form's 8 pi^2 nu (Sec. 3.1's viscous cases; 200 steps reach only t = 0.118)
    for kappa in (1.6, 2.0):
        case = inputs.tgv2d(nx=50, kappa=kappa)
        sim, nnz, oh = _eulerian_case(api, ctx, case, api.SPH_FP64)
        nsteps = int(math.ceil(1.0 / case["dt"]))
        ts, amp = [], []
        done = 0
        while True:
            _, v = sim.fields()
            ts.append(done * case["dt"])
            amp.append(math.sqrt(2.0 * float(torch.mean(torch.sum(v * v, dim=0)))) / case["U"])
            if done >= nsteps:
                break
            k = min(50, nsteps - done)
            sim.step(k)
            done += k
        ts, amp = np.array(ts), np.array(amp)
        rate = -np.polyfit(ts, np.log(amp), 1)[0]
        t = done * case["dt"]
        _, v = sim.fields()
        exact = torch.tensor(inputs.tgv2d_exact_velocity(case["pos"][:, oh], case["U"], case["nu"], t),
                             device=ctx.device)
        out["kappa_%.1f" % kappa]["t1"] = {
            "t": t, "steps": done, "decay_rate_fit": rate, "decay_rate_exact": case["decay_rate"],
            "decay_rate_rel_err": rate / case["decay_rate"] - 1.0,
            "l2_v_vs_closed_form": float(torch.linalg.norm(v - exact) / torch.linalg.norm(exact))}
    out["matched_accuracy_t1"] = (out["kappa_1.6"]["t1"]["l2_v_vs_closed_form"]
                                  <= 1.1 * out["kappa_2.0"]["t1"]["l2_v_vs_closed_form"])
    out["matched_accuracy_criterion"] = "L2(v - closed form) at 1.6h <= 1.1 x the same at 2h, same dp"
    return out


def _bench_plate_accuracy(api, inputs, ctx, every=100):
    """The headline plate at 1.6h and 2h (float32 + Kahan, tile plan) run to 0.9 of the
    Euler-Bernoulli first-mode period (the large-amplitude oscillation is slower than the
    linear estimate): the tip deflection history (mean u_y over the tip face), its first
    maximum and zero crossing (period = twice the crossing time), against the
    Euler-Bernoulli plate estimate, and the energy drift (float64 reduction)."""
    import torch
    c16 = inputs.plate(dp=0.001, kappa=1.6)
    L, t = 0.2, 0.02
    E, nu, rho0 = 2.0e6, 0.3975, c16["rho0"]
    # first bending mode of a clamped-free plate strip (plate modulus E / (1 - nu^2))
    omega = 1.875104068711961 ** 2 * math.sqrt(E * t * t / (12.0 * rho0 * (1.0 - nu * nu))) / (L * L)
    T_eb = 2.0 * math.pi / omega
    out = {"workload": "cantilever plate, dp=1 mm (816,000 particles), neo-Hookean, float32 + Kahan on the tile "
                       "plan, run to 0.9 of the Euler-Bernoulli first period; tip = the last layer (x = L - dp/2)",
           "euler_bernoulli_period_s": T_eb, "euler_bernoulli_tip_amplitude_m": 0.05 * c16["c0"] / omega}
    curves = {}
    for kappa in (1.6, 2.0):
        s = _setup_plate(api, inputs, ctx, kappa)
        sol = _solid(api, ctx, s, api.SPH_FP32_KAHAN)
        dt = s["c"]["dt"]
        nsteps = int(math.ceil(0.9 * T_eb / dt))
        tip = s["r0"][0] > L - 0.001          # the last layer, x = L - dp/2
        e0 = sol.energy()
        ts, uy = [], []
        done = 0
        t0 = time.perf_counter()
        while True:
            x, _, _ = sol.fields()
            ts.append(done * dt)
            uy.append(float(torch.mean((x[1] - s["r0"][1])[tip])))
            if done >= nsteps:
                break
            k = min(every, nsteps - done)
            sol.step(k)
            done += k
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        e1 = sol.energy()
        ts, uy = np.array(ts), np.array(uy)
        imax = int(np.argmax(uy))
        cross = None
        for k in range(imax, len(uy) - 1):
            if uy[k] > 0.0 >= uy[k + 1]:
                cross = ts[k] + (ts[k + 1] - ts[k]) * uy[k] / (uy[k] - uy[k + 1])
                break
        curves[kappa] = uy
        out["kappa_%.1f" % kappa] = {
            "steps": done, "t_end_s": done * dt, "wall_s_with_readbacks": wall,
            "tip_max_m": float(uy[imax]), "t_tip_max_s": float(ts[imax]),
            "t_zero_crossing_s": cross, "period_estimate_s": None if cross is None else 2.0 * cross,
            "period_vs_euler_bernoulli": None if cross is None else 2.0 * cross / T_eb,
            "energy_start_J": list(e0), "energy_end_J": list(e1),
            "energy_drift_rel": (sum(e1) - sum(e0)) / sum(e0)}
        del sol, s
        torch.cuda.empty_cache()
    a, b = curves[1.6], curves[2.0]
    m = min(len(a), len(b))
    out["tip_curve_rel_diff_max"] = float(np.max(np.abs(a[:m] - b[:m])) / np.max(np.abs(b[:m])))
    p16, p20 = out["kappa_1.6"]["period_estimate_s"], out["kappa_2.0"]["period_estimate_s"]
    out["period_rel_diff_tw_vs_sw"] = None if (p16 is None or p20 is None) else p16 / p20 - 1.0
    out["matched_accuracy_criterion"] = ("tip deflection curves of 1.6h and 2h within 5 % of the 2h amplitude and "
                                         "their periods within 2 %")
    out["matched_accuracy"] = bool(out["tip_curve_rel_diff_max"] <= 0.05 and p16 is not None and p20 is not None
                                   and abs(p16 / p20 - 1.0) <= 0.02)
    return out


def _bench_batched(api, inputs, ctx, steps, peak):
    """64 uneven 2D Taylor-Green cases (64^2 .. 1024^2, Re in {100, 1000}) in one persistent launch per pass."""
    from paper_2405_05155_gb300 import batch
    from paper_2405_05155_gb300._lib import SPH_TIMER_BATCH_STEP
    cases = inputs.batched_tgv2d(seed=0, ncases=64)
    b = batch.EulerianBatch(ctx, cases)
    lanes, block, _ = b.autotune(trial_steps=3)
    b.step(10)
    ctx.timing(True, every=TIMER_EVERY)
    ms = _event_ms(lambda: b.step(steps))
    tstep, nstep = ctx.timer(SPH_TIMER_BATCH_STEP)
    ctx.timing(False)
    per_step_bytes = 2 * (b.ntotal * (8 + 64 + 16) + 4 * b.nnz)
    return {"workload": "64 independent 2D Taylor-Green cases, sides log-uniform 64..1024 (seed 0), "
                        "Re in {100,1000}, kappa=1.6, FP32+Kahan, persistent launch per pass, CUDA graph",
            "particles": b.ntotal, "nnz": b.nnz, "ms_per_step": ms / steps,
            "pair_interactions_per_s": 2 * b.nnz * steps / (ms * 1e-3), "lanes": lanes, "block": block,
            "roofline": _roof(per_step_bytes, tstep / max(nstep, 1), peak)}


def _bench_relax(api, inputs, ctx, steps, peak):
    """Laguerre-Gauss relaxation of the 8-sphere body at dp = 1/128 (float32 pair sums)."""
    from paper_2405_05155_gb300 import learned
    from paper_2405_05155_gb300._lib import SPH_TIMER_NEIGHBORS, SPH_TIMER_RELAX_ACCEL, SPH_TIMER_RELAX_UPDATE
    b, prm, pos, vol = learned.body_on_device(ctx, 0, 1.0 / 128.0)
    n = pos.shape[1]
    skin = 0.2
    ctx.set_relax_skin(skin)
    r0 = api.relax_residual(ctx, prm, pos, vol)
    api.relax_step(ctx, prm, pos, vol, 3)
    ms = _event_ms(lambda: api.relax_step(ctx, prm, pos, vol, steps))
    # the same call once more with per-kernel events around every launch, for the breakdown
    ctx.timing(True)
    api.relax_step(ctx, prm, pos, vol, steps)
    tn, nn = ctx.timer(SPH_TIMER_NEIGHBORS)
    ta, na = ctx.timer(SPH_TIMER_RELAX_ACCEL)
    tu, nu = ctx.timer(SPH_TIMER_RELAX_UPDATE)
    ctx.timing(False)
    # the list-free form: a cell sweep every step
    ctx.set_relax_skin(0.0)
    sweep_steps = 10
    ms_sweep = _event_ms(lambda: api.relax_step(ctx, prm, pos, vol, sweep_steps)) / sweep_steps
    ctx.set_relax_skin(skin)
    r1 = api.relax_residual(ctx, prm, pos, vol)
    # pairs per step: the LG neighbour count of the current positions
    rp, col = api.build_neighbors(ctx, b["domain"], pos)
    nnz = int(col.numel())
    # walk: own records (32 B in, 16 B out) and the list stream, ~(2.2/2)^3 entries per pair
    list_entries = nnz * ((2.0 + skin) / 2.0) ** 3
    acc_bytes = n * (32 + 16 + 4) + 4 * list_entries
    return {"workload": "Laguerre-Gauss relaxation, union of 8 seeded spheres (seed 0), dp=1/128, h=1.3dp, "
                        "cut-off 2h, jitter 0.25dp, FP32+Kahan pair sums, list of cut-off 2h + %.1fh rebuilt "
                        "when twice the largest displacement exceeds the skin" % skin,
            "particles": n, "nnz": nnz, "ms_per_step": ms / steps,
            "pair_interactions_per_s": nnz * steps / (ms * 1e-3),
            "list_builds_per_%d_steps" % steps: nn,
            "ms_breakdown": {"list_build": tn / max(nn, 1), "accel_pass": ta / max(na, 1),
                             "update": tu / max(nu, 1)},
            "cell_sweep_every_step_ms_per_step": ms_sweep,
            "residual_lg": [r0[0], r1[0]], "residual_tw": [r0[1], r1[1]], "steps": 3 + 2 * steps + sweep_steps,
            "roofline_accel_pass": _roof(acc_bytes, ta / max(na, 1), peak)}


def _bench_error_analysis(api, inputs, ctx, relax_steps=1000):
    """Sec. 2.3.3: the L2 errors (Eq. 10) of the SPH summation of f = 1 and of the weak-form
    df/dx of f = exp(-x^2/0.1) on a circle of diameter 2 (h = 1.3 dp), over the particles
    at least 2h inside the surface, for the lattice and the Wendland- and Laguerre-Gauss-
    relaxed distributions, standard (2h) and truncated (1.6h) Wendland kernels, with and
    without the correction matrix.  Everything on the GPU (float64)."""
    import math
    import torch
    dev = ctx.device
    table = {}
    approx_ms = None
    start = torch.cuda.Event(enable_timing=True)
    stop = torch.cuda.Event(enable_timing=True)
    start.record()
    for nres in (10, 20, 40):
        dp = 2.0 / nres
        lat = inputs.circle_body(dp)
        jit = inputs.circle_body(dp, jitter=0.25, seed=0)
        dists = {"lattice": torch.tensor(lat["pos"], dtype=torch.float64, device=dev)}
        res = {}
        for name, kernel in (("wendland_relaxed", api.SPH_WENDLAND_C2), ("laguerre_gauss_relaxed",
                                                                         api.SPH_LAGUERRE_GAUSS)):
            pos = torch.tensor(jit["pos"], dtype=torch.float64, device=dev)
            vol = torch.tensor(jit["vol"], dtype=torch.float64, device=dev)
            prm = api.relax_params(jit["domain"], jit["spheres"], dp, precision=api.SPH_FP64, kernel=kernel)
            r0 = api.relax_residual(ctx, prm, pos, vol)
            api.relax_step(ctx, prm, pos, vol, relax_steps)
            r1 = api.relax_residual(ctx, prm, pos, vol)
            dists[name] = pos
            res[name] = {"residual_lg": [r0[0], r1[0]], "residual_tw": [r0[1], r1[1]]}
        row = {}
        for name, pos in dists.items():
            n = pos.shape[1]
            vol = torch.full((n,), dp * dp, dtype=torch.float64, device=dev)
            x = pos[0]
            interior = torch.sqrt(pos[0] ** 2 + pos[1] ** 2) - 1.0 < -2.0 * 1.3 * dp
            f_exp = torch.exp(-x * x / 0.1)
            dfdx = -2.0 * x / 0.1 * f_exp
            ones = torch.ones(n, dtype=torch.float64, device=dev)
            entry = {"particles": n, "interior": int(interior.sum())}
            for label, kappa in (("SW", 2.0), ("TW", 1.6)):
                d = dict(lat["domain"])
                d["kappa"] = kappa
                rp, col = api.build_neighbors(ctx, d, pos)
                B, _, nfb = api.kgc(ctx, d, pos, vol, rp, col)
                s1, _ = api.field_approx(ctx, d, pos, vol, rp, col, ones)
                _, g = api.field_approx(ctx, d, pos, vol, rp, col, f_exp)
                _, gB = api.field_approx(ctx, d, pos, vol, rp, col, f_exp, B=B)
                if nres == 40 and label == "TW" and name == "laguerre_gauss_relaxed":
                    approx_ms = _event_ms(lambda: api.field_approx(ctx, d, pos, vol, rp, col, f_exp, B=B))

                def l2(ref, app):
                    ref, app = ref[interior], app[interior]
                    return float(torch.sqrt(torch.sum((ref - app) ** 2) / torch.sum(ref * ref)))

                entry[label + "_f1_without_B"] = l2(ones, s1)
                entry[label + "_dfdx_without_B"] = l2(dfdx, g[0])
                entry[label + "_dfdx_with_B"] = l2(dfdx, gB[0])
                entry[label + "_kgc_fallbacks"] = nfb
            if name in res:
                entry.update(res[name])
            row[name] = entry
        table["dp=D/%d" % nres] = row
    stop.record()
    torch.cuda.synchronize()
    return {"workload": "error analysis of Sec. 2.3.3: circle D = 2, dp = D/10, D/20, D/40, h = 1.3 dp; lattice and "
                        "distributions relaxed %d steps (float64) with the standard Wendland or the Laguerre-Gauss "
                        "kernel from a lattice jittered by U(-dp/4, dp/4) (seed 0); L2 of Eq. 10 over particles "
                        "with phi < -2h" % relax_steps,
            "table": table,
            "paper_table1_f1_dp_D10": {"lattice": {"SW": 0.010, "TW": 0.006},
                                       "wendland_relaxed": {"SW": 0.034, "TW": 0.028},
                                       "laguerre_gauss_relaxed": {"SW": 0.037, "TW": 0.031}},
            "field_approx_ms_dp_D40": approx_ms,
            "total_ms": start.elapsed_time(stop)}


def _bench_dsl(api, inputs, ctx, t_end=1.2):
    """The inviscid double shear layer of Sec. 5 (unit periodic square, float32 + Kahan, tile
    plan): at dp = 1/128 the whole run to t = 1.2 with the truncated (1.6h) and standard (2h)
    kernels, their ratio alpha (the paper: 0.59 on one CPU core), the difference of the two
    velocity fields at the end and the vorticity range (weak-form gradients with B on the
    GPU); at dp = 1/1024 (1M particles) the ms per step of both."""
    import torch
    out = {"workload": "inviscid double shear layer (rho = 1/30, delta = 0.05), unit periodic square, h = 1.3 dp, "
                       "c0 = 10, acoustic Riemann two-pass step, float32 + Kahan on the tile plan"}
    for nx in (128, 1024):
        row = {}
        fields = {}
        for kappa in (2.0, 1.6):
            case = inputs.double_shear_layer(nx, kappa=kappa)
            sim, nnz, _ = _eulerian_case(api, ctx, case, api.SPH_FP32_KAHAN)
            dt = case["dt"]
            steps = int(round(t_end / dt)) if nx == 128 else 200
            sim.step(3)
            sim, _, order = _eulerian_case(api, ctx, case, api.SPH_FP32_KAHAN)
            ms = _event_ms(lambda: sim.step(steps))
            key = "kappa_%.1f" % kappa
            row[key] = {"particles": case["pos"].shape[1], "nnz": nnz, "steps": steps,
                        "ms_per_step": ms / steps, "pair_interactions_per_s": 2 * nnz * steps / (ms * 1e-3)}
            if nx == 128:
                row[key]["run_to_t_ms"] = ms
                _, v = sim.fields()
                d = dict(case["domain"])
                _, gx = api.field_approx(ctx, d, sim.pos, sim.vol, sim.row_ptr, sim.col, v[0].contiguous(), B=sim.B)
                _, gy = api.field_approx(ctx, d, sim.pos, sim.vol, sim.row_ptr, sim.col, v[1].contiguous(), B=sim.B)
                omega = gy[0] - gx[1]
                row[key]["vorticity_min_max_at_t_end"] = [float(omega.min()), float(omega.max())]
                # back to the input order (the cell order depends on the cut-off)
                inv = torch.empty(len(order), dtype=torch.int64, device=v.device)
                inv[torch.as_tensor(order, device=v.device)] = torch.arange(len(order), device=v.device)
                fields[kappa] = v[:, inv].clone()
            del sim
            torch.cuda.empty_cache()
        row["alpha_TW_over_SW"] = row["kappa_1.6"]["ms_per_step"] / row["kappa_2.0"]["ms_per_step"]
        if fields:
            a, b = fields[1.6], fields[2.0]
            row["rel_l2_TW_vs_SW_velocity_at_t_end"] = float(torch.linalg.norm(a - b) / torch.linalg.norm(b))
            row["t_end"] = t_end
        out["dp=1/%d" % nx] = row
    out["paper"] = {"dp=1/128": {"cpu_s_SW": 29.99, "cpu_s_TW": 17.83, "alpha": 0.59}}
    return out


def _bench_columns(api, inputs, ctx, steps=200):
    """The twisting and bending columns of Sec. 5 (total-Lagrangian, neo-Hookean, float32 +
    Kahan on the tile plan): ms per step with the truncated (1.6h) and standard (2h) kernels
    at the paper's resolutions and their ratio alpha (the paper's Tables: CPU wall-clock
    ratios); and, at the coarsest resolutions, a stability run of each column to its
    end time with both kernels."""
    import torch
    out = {"workload": "3D columns, side 1 m x height 6 m, clamped base (3 layers), rho0 = 1100, E = 17 MPa, "
                       "h = 1.15 dp; twisting: nu = 0.499, Omega = 105 sin(pi y / 12) rad/s about the axis; "
                       "bending: nu = 0.45, v = 10 (sqrt 3 / 2, 1/2, 0) m/s",
           "paper_alpha": {"twisting": {"1/10": 0.67, "1/20": 0.68, "1/30": 0.64},
                           "bending": {"1/6": 0.69, "1/12": 0.47, "1/24": 0.56}}}
    for kind, sides, t_end in (("twisting", (10, 20, 30), 0.0909), ("bending", (6, 12, 24), 0.5)):
        rows = {}
        for n_side in sides:
            row = {}
            for kappa in (2.0, 1.6):
                c = inputs.column(kind, n_side, kappa=kappa)
                s = _setup_solid(api, ctx, c)
                sol = _solid(api, ctx, s, api.SPH_FP32_KAHAN)
                sol.step(3)
                ms = _event_ms(lambda: sol.step(steps))
                key = "kappa_%.1f" % kappa
                row[key] = {"particles": s["n"], "nnz": s["nnz"], "ms_per_step": ms / steps,
                            "pair_interactions_per_s": 2 * s["nnz"] * steps / (ms * 1e-3), "dt": c["dt"]}
                if n_side == sides[0]:
                    # the whole run to t_end from the initial state
                    sol = _solid(api, ctx, s, api.SPH_FP32_KAHAN)
                    nsteps = int(round(t_end / c["dt"]))
                    ms_run = _event_ms(lambda: sol.step(nsteps))
                    x, v, H = sol.fields()
                    top = s["r0"][1] >= s["r0"][1].max() - 1e-9
                    disp = (x - s["r0"])[:, top].mean(dim=1)
                    row[key].update({"t_end": t_end, "run_steps": nsteps, "run_ms": ms_run,
                                     "finite": bool(torch.isfinite(x).all() and torch.isfinite(v).all()),
                                     "top_mean_displacement_m": [float(u) for u in disp],
                                     "max_speed": float(torch.sqrt((v * v).sum(0)).max())})
                del sol
                torch.cuda.empty_cache()
            row["alpha_TW_over_SW"] = row["kappa_1.6"]["ms_per_step"] / row["kappa_2.0"]["ms_per_step"]
            rows["1/%d" % n_side] = row
        out[kind] = rows
    return out


def _compressible_case(api, ctx, c, precision):
    import torch
    d = c["domain"]
    dev = torch.device("cuda", torch.cuda.current_device())
    pos = torch.as_tensor(c["pos"], dtype=torch.float64, device=dev)
    order = api.cell_order(ctx, d, pos)
    pos = pos[:, order].contiguous()
    vol = torch.as_tensor(c["vol"], dtype=torch.float64, device=dev)[order].contiguous()
    rp, col = api.build_neighbors(ctx, d, pos)
    B, _, _ = api.kgc(ctx, d, pos, vol, rp, col)
    oh = order.cpu().numpy()
    sim = api.Compressible(ctx, d, pos, vol, B, rp, col, c["rho"][oh], c["mom"][:, oh], c["E"][oh], c["dt"],
                           gamma=c["gamma"], precision=precision)
    return sim, int(col.numel()), oh


def _comp_bytes(n, nnz, dim):
    """Algorithmic bytes of one float32 compressible step, by the rule of the other planned
    passes: per pair the int32 neighbour index; per particle its row offset (8 B), its
    record (32 B), the float64 state read and written (2 x (dim + 2) x 8 B) and the next
    record written (32 B).  The neighbours' records stay in L2 across the pairs that read
    them; the plan's precomputed pair geometry (16 B more per pair in 2D, 28 B in 3D) is a
    trade of arithmetic for bytes, not counted (ncu's DRAM bytes show it)."""
    return nnz * 4 + n * (8 + 32 + 2 * (dim + 2) * 8 + 32)


def _bench_compressible(api, inputs, ctx, peak, steps=200):
    """Compressible Riemann SPH (Sec. 3.1, limited HLLC): ms per step of a 4096 x 64 Sod
    strip (262,144 particles) with the truncated (1.6h) and standard (2h) kernels and their
    ratio alpha, in the float32 form (the plan of fixed pair geometry, one kernel per step)
    and the float64 form; and at 1024 x 8 the whole run to t = 0.1 with both kernels and
    the relative L1 difference of their density fields."""
    import numpy as np
    import torch
    out = {"workload": "2D Sod strip periodic in x and y (two mirrored Sod tubes), ideal gas gamma = 1.4, "
                       "h = 1.3 dp, dt = 0.2 h / 2.5, forward Euler, HLLC with the dissipation limiter (eta = 1)"}
    forms = (("fp32_kahan", api.SPH_FP32_KAHAN), ("fp64", api.SPH_FP64))
    for nx, ny, full in ((4096, 64, False), (1024, 8, True)):
        row = {}
        for fname, prec in forms:
            frow = {}
            rho_end = {}
            for kappa in (2.0, 1.6):
                c = inputs.sod_strip(nx=nx, ny=ny, kappa=kappa)
                sim, nnz, oh = _compressible_case(api, ctx, c, prec)
                nsteps = int(round(0.1 / c["dt"])) if full else (steps if prec == api.SPH_FP64 else 10 * steps)
                key = "kappa_%.1f" % kappa
                by_lanes = {}
                if prec == api.SPH_FP32_KAHAN and not full:
                    # launch shape: lanes per row (results differ by float32 rounding only)
                    for lanes in (1, 2, 4, 8):
                        ctx.set_lanes(api.SPH_PASS_COMPRESSIBLE, lanes)
                        sim.step(3)
                        by_lanes[lanes] = _event_ms(lambda: sim.step(steps)) / steps
                    ctx.set_lanes(api.SPH_PASS_COMPRESSIBLE, min(by_lanes, key=by_lanes.get))
                if not full:
                    sim.step(3)
                ms = _event_ms(lambda: sim.step(nsteps))
                frow[key] = {"particles": int(sim.n), "nnz": nnz, "steps": nsteps, "ms_per_step": ms / nsteps,
                             "pair_evaluations_per_s": nnz * nsteps / (ms * 1e-3)}
                if by_lanes:
                    frow[key]["lanes"] = ctx.get_lanes(api.SPH_PASS_COMPRESSIBLE)
                    frow[key]["ms_per_step_by_lanes"] = by_lanes
                if prec == api.SPH_FP32_KAHAN and not full:
                    frow[key]["roofline"] = _roof(_comp_bytes(sim.n, nnz, 2), ms / nsteps, peak)
                    frow[key]["roofline"]["kernel"] = "k_comp32"
                if full:
                    rho = np.empty(sim.n)
                    rho[oh] = sim.rho.cpu().numpy()          # back to the input order
                    rho_end[kappa] = rho
                    frow[key]["run_to_t_ms"] = ms
                    frow[key]["rho_min_max_at_t_end"] = [float(rho.min()), float(rho.max())]
                del sim
                torch.cuda.empty_cache()
            frow["alpha_TW_over_SW"] = frow["kappa_1.6"]["ms_per_step"] / frow["kappa_2.0"]["ms_per_step"]
            if rho_end:
                a, b = rho_end[1.6], rho_end[2.0]
                frow["rel_l1_TW_vs_SW_density_at_t_0.1"] = float(np.sum(np.abs(a - b)) / np.sum(np.abs(b)))
            row[fname] = frow
        out["%dx%d" % (nx, ny)] = row
    return out


def _bench_mlp(api, inputs, ctx, peak_tflops):
    """BF16 tensor-core MLP: proposal forward over a 2.2M-row feature set, and training steps."""
    import torch
    from paper_2405_05155_gb300 import learned
    b, prm, pos, vol = learned.body_on_device(ctx, 1, 1.0 / 128.0)
    feats = api.mlp_features(ctx, prm, pos)
    rows = feats.shape[0]
    params = torch.tensor(inputs.mlp_init(0), dtype=torch.float32, device=ctx.device)
    api.mlp_forward(ctx, params, feats)
    ms_mma = _event_ms(lambda: [api.mlp_forward(ctx, params, feats) for _ in range(5)]) / 5
    api.mlp_forward_tc(ctx, params, feats)
    ms = _event_ms(lambda: [api.mlp_forward_tc(ctx, params, feats, check=False) for _ in range(20)]) / 20
    y_tc = api.mlp_forward_tc(ctx, params, feats)
    y_mma = api.mlp_forward(ctx, params, feats)
    diff = float(torch.linalg.norm(y_tc - y_mma) / torch.linalg.norm(y_mma))
    flops = 2.0 * rows * (128 * 128 * 3 + 128 * 3)
    tr = api.MLPTrainer(ctx, inputs.mlp_init(0))
    x = feats[:4096].contiguous()
    t = torch.zeros((4096, 3), dtype=torch.float32, device=ctx.device)
    tr.step(x, t)
    ms_tr = _event_ms(lambda: [tr.step(x, t) for _ in range(20)]) / 20
    tflops = flops / (ms * 1e-3) / 1e12
    return {"workload": "128-128-128-128-3 GELU MLP, BF16 operands, FP32 accumulate; fused forward on tcgen05 "
                        "(TMEM accumulators) over the features of a dp=1/128 body; mma.sync reference forward and an Adam "
                        "step at batch 4096 (training path)",
            "rows": rows, "forward_ms": ms, "forward_tflops": tflops, "forward_mma_sync_ms": ms_mma,
            "rel_l2_tcgen05_vs_mma_sync": diff, "train_step_ms_batch4096": ms_tr,
            "roofline": {"bound": "tensor", "kernel": "k_mlp_forward_tc", "achieved": tflops, "peak": peak_tflops,
                         "unit": "TFLOP/s", "frac": tflops / peak_tflops}}


def _bench_relax_learned(api, inputs, ctx, train_bodies=200, train_steps=4000, target_steps=(50, 200)):
    """The learned proposal at the relaxation configuration's scale, all through the C ABI:
    training data from plain trajectories of `train_bodies` seeded bodies at dp = 1/40
    (sph_relax_samples: 500 steps, a snapshot every 50), Adam on device-drawn minibatches of
    4096 (sph_mlp_train), then wall-clock to a residual target on the dp = 1/128 body of seed
    0 (sph_relax_run): plain float64, plain float32 and float32 with the proposal.  The
    target is the residual plain float32 relaxation reaches after `target_steps` steps."""
    import time
    import torch
    from paper_2405_05155_gb300 import learned
    t0 = time.perf_counter()
    feats, targets = learned.training_set(ctx, range(train_bodies), 1.0 / 40.0, steps=500, every=50)
    torch.cuda.synchronize()
    t_data = time.perf_counter() - t0
    rows = int(feats.shape[0])
    t0 = time.perf_counter()
    trainer, losses = learned.train(ctx, feats, targets, steps=train_steps, batch=4096, lr=1e-3, seed=0,
                                    log_every=1000)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    del feats, targets
    torch.cuda.empty_cache()
    b, prm32, pos0, vol = learned.body_on_device(ctx, 0, 1.0 / 128.0)
    prm64 = api.relax_params(b["domain"], b["spheres"], b["dp"], precision=api.SPH_FP64, n=pos0.shape[1])
    # the judge: the residual from float32 pair sums (float64 reduction), every 10 plain steps;
    # the target is what plain float32 relaxation reaches after target_steps steps, judged
    # the same way
    r_start = api.relax_residual_fp32(ctx, prm32, pos0, vol)[0]
    judge_ms = _event_ms(lambda: api.relax_residual_fp32(ctx, prm32, pos0, vol))
    judge64_ms = _event_ms(lambda: api.relax_residual(ctx, prm32, pos0, vol))
    propose_ms = _event_ms(lambda: api.relax_propose(ctx, prm32, trainer.params, pos0.clone()))
    by_target = {}
    for ts_ in target_steps:
        ref = pos0.clone()
        api.relax_run(ctx, prm32, ref, vol, 0.0, ts_, check_every=ts_, judge=api.SPH_FP32_KAHAN)
        target = api.relax_residual_fp32(ctx, prm32, ref, vol)[0]
        del ref
        arms = {}
        for name, prm, proposal in (("plain_fp32", prm32, None), ("learned_fp32", prm32, trainer.params),
                                    ("plain_fp64", prm64, None)):
            p = pos0.clone()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            out = api.relax_run(ctx, prm, p, vol, target, 20 * ts_, proposal=proposal, applications=3,
                                plain_between=10, check_every=10, judge=api.SPH_FP32_KAHAN)
            torch.cuda.synchronize()
            out["ms"] = (time.perf_counter() - t0) * 1e3
            arms[name] = out
            del p
        by_target["plain_fp32_%d_steps" % ts_] = {
            "residual_target": target, "arms": arms,
            "speedup_learned_vs_plain_fp32": arms["plain_fp32"]["ms"] / arms["learned_fp32"]["ms"],
            "speedup_learned_vs_plain_fp64": arms["plain_fp64"]["ms"] / arms["learned_fp32"]["ms"]}
    return {"workload": "learned relaxation proposal: trained on %d seeded 8-sphere bodies at dp=1/40 (%d samples, "
                        "snapshots every 50 of 500 plain steps), Adam lr 1e-3, batch 4096, %d steps; applied to the "
                        "dp=1/128 body of seed 0 (%d particles); residual targets = what plain float32 relaxation "
                        "reaches after %s steps; residual checked every 10 plain steps"
                        % (train_bodies, rows, train_steps, int(pos0.shape[1]), "/".join(str(x) for x in target_steps)),
            "training_data_s": t_data, "training_s": t_train, "loss": losses, "residual_start": r_start,
            "judge": "sph_relax_residual_fp32 (float32 pair sums, float64 reduction)",
            "judge_ms": judge_ms, "float64_residual_ms": judge64_ms, "propose_ms": propose_ms,
            "targets": by_target}


# --------------------------------------------------------------------------- arms
def run_reference(args):
    rank, world, _ = _dist_info()
    if rank != 0:
        return 0
    cb = _cpu_baseline(steps_cap_s=max(3.0, min(60.0, 1.0 * args.steps / 100.0 + 8.0)))
    line = {"impl": "reference", "metric": METRIC, "value": cb["value"], "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": cb["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "reference": "float64 CPU oracle (oracle/), "
                                            "bounded sample of the same workload"},
            "cpu_baseline": {"value": cb["value"], "unit": UNIT, "cores": cb["cores"], "kind": "oracle",
                             "sample": cb["sample"], "single_core": cb["single_core"]},
            "e2e": {"value": cb["value"], "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def run_gpu(args):
    import torch
    rank, world, local = _dist_info()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", init_method="env://")
    else:
        torch.cuda.set_device(0)
    from paper_2405_05155_gb300 import api, inputs
    from paper_2405_05155_gb300._lib import SPH_TIMER_TL_DEFORM, SPH_TIMER_TL_MOMENTUM, SPH_TIMER_TL_STRESS
    ctx = api.Context(torch.cuda.current_device())
    K, W = args.steps, args.warmup
    if args.no_l2_persist:
        ctx.set_l2_persist(False)
    if args.pipe:
        ctx.set_tile_pipeline({"stream": api.SPH_PIPE_STREAM, "persistent": api.SPH_PIPE_PERSISTENT,
                               "bulk": api.SPH_PIPE_BULK, "geom": api.SPH_PIPE_GEOM}[args.pipe])

    if args.profile == "relax":
        from paper_2405_05155_gb300 import learned
        b, prm, pos, vol = learned.body_on_device(ctx, 0, 1.0 / 128.0)
        api.relax_step(ctx, prm, pos, vol, W + K)
        torch.cuda.synchronize()
        print(json.dumps({"profile": "relax", "particles": int(pos.shape[1]), "steps": W + K}))
        ctx.close()
        return 0
    if args.profile == "mlp":
        g = torch.Generator(device="cpu").manual_seed(0)
        feats = (0.8 * torch.randn((args.mlp_rows, 128), generator=g)).to(ctx.device)
        feats[:, 97:] = 0.0
        params = torch.tensor(inputs.mlp_init(0), dtype=torch.float32, device=ctx.device)
        for _ in range(W + K):
            api.mlp_forward_tc(ctx, params, feats, check=False)
        torch.cuda.synchronize()
        print(json.dumps({"profile": "mlp", "rows": args.mlp_rows, "launches": W + K}))
        ctx.close()
        return 0
    if args.profile == "comp":
        c = inputs.sod_strip(nx=args.comp_nx, ny=64, kappa=args.kappa)
        if args.lanes:
            ctx.set_lanes(api.SPH_PASS_COMPRESSIBLE, args.lanes)
        sim, nnz, _ = _compressible_case(api, ctx, c, api.SPH_FP32_KAHAN)
        sim.step(W + K)
        torch.cuda.synchronize()
        print(json.dumps({"profile": "comp", "particles": int(sim.n), "nnz": nnz, "steps": W + K}))
        del sim
        ctx.close()
        return 0
    if args.profile == "eu3d":
        case = inputs.tgv3d(n=args.eu_n, kappa=args.kappa)
        sim, nnz, _ = _eulerian_case(api, ctx, case, api.SPH_FP32_KAHAN, tiles=not args.no_tiles)
        sim.step(W + K)
        torch.cuda.synchronize()
        print(json.dumps({"profile": "eu3d", "n": args.eu_n, "kappa": args.kappa, "nnz": nnz, "steps": W + K}))
        ctx.close()
        return 0
    if args.profile:
        # profiling driver: the headline workload only (setup, then W + K float32 steps)
        s = _setup_plate(api, inputs, ctx, args.kappa)
        if args.lanes:
            ctx.set_lanes(api.SPH_PASS_TLSPH, args.lanes)
        sol = _solid(api, ctx, s, api.SPH_FP64 if args.profile == "fp64" else api.SPH_FP32_KAHAN,
                     tiles=not args.no_tiles)
        sol.step(W + K)
        torch.cuda.synchronize()
        print(json.dumps({"profile": args.profile, "kappa": args.kappa, "particles": s["n"], "nnz": s["nnz"],
                          "steps": W + K}))
        ctx.close()
        return 0

    # headline: truncated kernel (1.6h), float32 + Kahan, per-kernel timing on
    s16 = _setup_plate(api, inputs, ctx, 1.6)
    sol = _solid(api, ctx, s16, api.SPH_FP32_KAHAN, tiles=not args.no_tiles)
    planned = sol.plan is not None
    if args.lanes:
        ctx.set_lanes(api.SPH_PASS_TLSPH, args.lanes)
        lanes16 = args.lanes
    elif planned:
        lanes16 = 1          # the planned passes run one thread per row
    else:
        lanes16, _ = sol.autotune(10)
    sol.step(W)
    torch.cuda.synchronize()
    # per-kernel CUDA events inside the timed region around every TIMER_EVERY-th launch of
    # each pass (events around every launch cost about 9 us of a 0.17 ms step)
    ctx.timing(True, every=TIMER_EVERY)
    clocks = ClockSampler(torch.cuda.current_device()) if rank == 0 else None
    ms, clk = _time_steps(ctx, sol, K, 0, world, clocks)
    t_mom, n_mom = ctx.timer(SPH_TIMER_TL_MOMENTUM)
    t_def, n_def = ctx.timer(SPH_TIMER_TL_DEFORM)
    t_str, n_str = ctx.timer(SPH_TIMER_TL_STRESS)
    launches = sum(ctx.launches(k) for k in (SPH_TIMER_TL_MOMENTUM, SPH_TIMER_TL_DEFORM, SPH_TIMER_TL_STRESS))
    ctx.timing(False)
    ms_step = ms / K
    pairs_step = 2 * s16["nnz"]
    value = _sum_over_ranks(pairs_step * K, world) / (ms * 1e-3)

    # float32 vs float64 after the same W + K steps (matched error vs FP64)
    x32, v32, H32 = [t.clone() for t in sol.fields()]
    sol64 = _solid(api, ctx, s16, api.SPH_FP64)
    ms64, _ = _time_steps(ctx, sol64, K, W, world)
    x64, v64, H64 = sol64.fields()

    def rl2(a, b):
        return float(torch.linalg.norm(a - b) / torch.linalg.norm(b))
    l2 = {"v": rl2(v32, v64), "H": rl2(H32, H64), "u": rl2(x32 - s16["r0"], x64 - s16["r0"])}
    del sol64

    # standard kernel (2h), same precision
    s20 = _setup_plate(api, inputs, ctx, 2.0)
    sol20 = _solid(api, ctx, s20, api.SPH_FP32_KAHAN)
    lanes20 = args.lanes or (1 if sol20.plan is not None else sol20.autotune(10)[0])
    ctx.set_lanes(api.SPH_PASS_TLSPH, lanes20)
    ms20, _ = _time_steps(ctx, sol20, K, W, world)
    _, v20, H20 = sol20.fields()
    # in the input order of the particles (each cut-off has its own cell order)
    i16, i20 = s16["inv"], s20["inv"]
    tw_vs_sw = {"v": rl2(v32[:, i16], v20[:, i20]), "H": rl2(H32[:, i16], H20[:, i20]),
                "after_steps": K + W}
    del sol20

    # roofline of the dominant kernel
    mom_b, def_b = _alg_bytes_tl(s16["n"], s16["nnz"])
    avg_mom = t_mom / max(n_mom, 1)
    avg_def = t_def / max(n_def, 1)
    dominant = ("tl_deformation_pass", def_b, avg_def) if t_def >= t_mom else ("tl_momentum_pass", mom_b, avg_mom)
    peaks_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(peaks_path):
        peak = json.load(open(peaks_path))["hbm_gbs"]
        peak_src = "measured"
    else:
        peak, peak_src = 6800.0, "fallback"
    achieved = dominant[1] / (dominant[2] * 1e-3) / 1e9
    # ncu DRAM bytes (read + write) per launch of each planned TL pass on this workload, by
    # pipeline mode (profiles/tl_plate816k_fp32_launches.md: the geometry forms of both
    # passes, with their records persisting in L2, caches left as the program leaves them;
    # tl_pair_passes_plate816k_full.md: the entry forms of the stream mode)
    pipe = args.pipe or "geom"
    ncu_traffic = {("tl_momentum_pass", "geom"): 143.3e6, ("tl_momentum_pass", "stream"): 446.8e6,
                   ("tl_deformation_pass", "geom"): 198.0e6, ("tl_deformation_pass", "stream"): 509.1e6}
    traffic = args.traffic if args.traffic is not None else ncu_traffic.get((dominant[0], pipe))

    # end to end through the C ABI with the float64 state (x, v, F - I) in host memory:
    # every step reads it from the host, packs, steps, unpacks and writes it back.
    # (a) the state in mapped page-locked host buffers (sph_host_alloc): pack reads and
    #     unpack writes them in place over the host link (NVLink-C2C);
    # (b) the state in pinned host tensors, moved by cudaMemcpyAsync around pack/unpack.
    e2e_steps = min(K, args.e2e_steps)
    sol_e = _solid(api, ctx, s16, api.SPH_FP32_KAHAN)
    hx = sol_e.x.cpu().pin_memory()
    hv = sol_e.v.cpu().pin_memory()
    hH = sol_e.H.cpu().pin_memory()
    h2d = (hx.numel() + hv.numel() + hH.numel()) * 8
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)

    def _timed(body):
        torch.cuda.synchronize()
        _barrier(world)
        t0.record()
        for _ in range(e2e_steps):
            body()
        t1.record()
        torch.cuda.synchronize()
        return _max_over_ranks(t0.elapsed_time(t1), world)

    def _with_copies():
        sol_e.x.copy_(hx, non_blocking=True)
        sol_e.v.copy_(hv, non_blocking=True)
        sol_e.H.copy_(hH, non_blocking=True)
        sol_e.pack()
        sol_e.step(1)
        sol_e.unpack()
        hx.copy_(sol_e.x, non_blocking=True)
        hv.copy_(sol_e.v, non_blocking=True)
        hH.copy_(sol_e.H, non_blocking=True)

    e2e_copy_ms = _timed(_with_copies)
    mapped = [api.HostArray(t.shape) for t in (sol_e.x, sol_e.v, sol_e.H)]
    for m, t in zip(mapped, (hx, hv, hH)):
        m.t.copy_(t)
    sol_m = _solid(api, ctx, s16, api.SPH_FP32_KAHAN)
    sol_m.st.x, sol_m.st.v, sol_m.st.H = mapped[0].dev, mapped[1].dev, mapped[2].dev

    def _in_place():
        sol_m.pack()
        sol_m.step(1)
        sol_m.unpack()

    e2e_ms = _timed(_in_place)
    e2e_value = _sum_over_ranks(pairs_step * e2e_steps, world) / (e2e_ms * 1e-3)
    e2e_copy_value = _sum_over_ranks(pairs_step * e2e_steps, world) / (e2e_copy_ms * 1e-3)
    e2e_ok = all(bool(torch.isfinite(m.t).all()) for m in mapped)
    for m in mapped:
        m.close()
    # (c) the float32 form's own state (u = x - r0, v, F - I) in float32 mapped host
    #     buffers, written into the records by load32 and read back by store32 around
    #     each step: the same values the step keeps, half the bytes of (a)
    sol_f = _solid(api, ctx, s16, api.SPH_FP32_KAHAN)
    n16 = s16["n"]
    b32 = [api.HostArray((3, n16), torch.float32), api.HostArray((3, n16), torch.float32),
           api.HostArray((9, n16), torch.float32)]
    sol_f.store32(*b32)
    torch.cuda.synchronize()

    def _f32_state():
        sol_f.load32(*b32)
        sol_f.step(1)
        sol_f.store32(*b32)

    def _f32_fused():
        sol_f.step_host32(*b32, nsteps=1)

    # the headline e2e: one call per step, copies overlapped with the passes; and the
    # same state moved by the three separate calls
    e2e32_ms = _timed(_f32_fused)
    e2e32_value = _sum_over_ranks(pairs_step * e2e_steps, world) / (e2e32_ms * 1e-3)
    e2e32c_ms = _timed(_f32_state)
    e2e32c_value = _sum_over_ranks(pairs_step * e2e_steps, world) / (e2e32c_ms * 1e-3)
    h2d32 = sum(b.t.numel() for b in b32) * 4
    e2e32_ok = all(bool(torch.isfinite(b.t).all()) for b in b32)
    for b in b32:
        b.close()

    workloads = {}
    if not args.headline_only:
        peaks = json.load(open(peaks_path)) if os.path.exists(peaks_path) else {}
        bf16 = peaks.get("bf16_tflops", 1900.0)
        for name, fn in (("tgv3d_128", lambda: _bench_tgv3d(api, inputs, ctx, args.other_steps, peak)),
                         ("tgv2d_50_plain_fp64", lambda: _bench_tgv2d(api, inputs, ctx)),
                         ("plate_matched_accuracy", lambda: _bench_plate_accuracy(api, inputs, ctx)),
                         ("batched_64_tgv2d", lambda: _bench_batched(api, inputs, ctx, args.other_steps, peak)),
                         ("relax_8spheres_dp128", lambda: _bench_relax(api, inputs, ctx, 50, peak)),
                         ("error_analysis_circle", lambda: _bench_error_analysis(api, inputs, ctx)),
                         ("double_shear_layer", lambda: _bench_dsl(api, inputs, ctx)),
                         ("columns", lambda: _bench_columns(api, inputs, ctx)),
                         ("compressible_sod", lambda: _bench_compressible(api, inputs, ctx, peak)),
                         ("mlp_proposal", lambda: _bench_mlp(api, inputs, ctx, bf16)),
                         ("relax_learned_8spheres_dp128", lambda: _bench_relax_learned(api, inputs, ctx))):
            if args.rows and name not in args.rows.split(","):
                continue
            # each row with the whole L2: the persisting lines of the rows before turned back
            # to normal (off, then on again for the rows that gather records)
            ctx.set_l2_persist(False)
            ctx.set_l2_persist(not args.no_l2_persist)
            try:
                workloads[name] = fn()
            except Exception as exc:      # report, do not hide: the headline line still prints
                workloads[name] = {"error": "%s: %s" % (type(exc).__name__, exc)}
            torch.cuda.empty_cache()

    if rank == 0:
        cb = _cpu_baseline(steps_cap_s=args.cpu_seconds) if world == 1 and not args.no_cpu else None
        ws = s16["n"] * (32 + 16 + 36 + 12 + 48 + 24) + 8 * (s16["n"] + 1) + 4 * s16["nnz"]
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
            "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "particles": s16["n"], "nnz": s16["nnz"],
                       "pairs_per_step": pairs_step, "kappa": 1.6, "kgc_fallbacks": s16["nfb"],
                       "l2_policy": "inputs larger than L2 (working set %.0f MB > 129 MB L2), no flush" % (ws / 2 ** 20),
                       "parallelism": "replicas" if world > 1 else "single GPU",
                       "lanes_per_particle": lanes16, "lanes_per_particle_2h": lanes20,
                       "launch_shape": ("tile plan: 128-row tiles, one thread per row, neighbours staged in "
                                        "shared memory; %s" % ("both passes evaluating grad0 W V0 from tile-relative "
                                                               "staged positions, the momentum pass as M_i S_i + "
                                                               "sum_j (V0_j M_j) g_ij (SPH_PIPE_GEOM)"
                                                               if pipe == "geom"
                                                               else "pipeline mode '%s'" % pipe))
                                       if planned else
                                       ("autotuned lanes (sph_autotune_tlsph)" if not args.lanes else "fixed lanes")},
            "kappa_2.0": {"ms_per_step": ms20 / K, "pair_interactions_per_s": 2 * s20["nnz"] * K / (ms20 * 1e-3),
                          "nnz": s20["nnz"]},
            "alpha_TW_over_SW": ms_step / (ms20 / K),
            "fp64": {"ms_per_step": ms64 / K, "pair_interactions_per_s": pairs_step * K / (ms64 * 1e-3)},
            "l2_fp32_vs_fp64": l2, "l2_tw_vs_sw": tw_vs_sw,
            "kernels_ms_avg": {"tl_momentum_pass": avg_mom, "tl_deformation_pass": avg_def,
                               "tl_stress_initial": t_str / max(n_str, 1)},
            "roofline": {"bound": "hbm", "kernel": dominant[0], "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic, "peak_source": peak_src,
                         "algorithmic_bytes_per_launch": dominant[1],
                         "by_kernel": {name: {"ms_per_launch": t, "achieved": b / (t * 1e-3) / 1e9,
                                              "frac": b / (t * 1e-3) / 1e9 / peak,
                                              "algorithmic_bytes_per_launch": b,
                                              "traffic": ncu_traffic.get((name, pipe))}
                                       for name, b, t in (("tl_momentum_pass", mom_b, avg_mom),
                                                          ("tl_deformation_pass", def_b, avg_def))}},
            "e2e": {"value": e2e32_value, "unit": UNIT, "steps": e2e_steps, "ms_per_step": e2e32_ms / e2e_steps,
                    "h2d_bytes_per_step": h2d32, "d2h_bytes_per_step": h2d32, "state_finite": e2e32_ok,
                    "state_form": "float32 (u = x - r0, v, F - I), 12 floats + 3x3 per particle; earlier "
                                  "lines of this file's history reported the float64 state under this key "
                                  "(now with_f64_state) and then the float32 state moved by three separate "
                                  "calls (now three_calls)",
                    "what": "per step, one call through the C ABI (sph_tlsph_step_host32): the float32 form's "
                            "state (u = x - r0, v, F - I) in float32 mapped page-locked host buffers "
                            "(sph_host_alloc) read in place over NVLink-C2C, one step, written back in place; "
                            "u read while the momentum pass runs and v written while the deformation pass "
                            "runs, on a second stream",
                    "three_calls": {"value": e2e32c_value, "ms_per_step": e2e32c_ms / e2e_steps,
                                    "h2d_bytes_per_step": h2d32, "d2h_bytes_per_step": h2d32,
                                    "what": "the same state moved by sph_tlsph_load32, sph_tlsph_step(1) and "
                                            "sph_tlsph_store32 in turn (no overlap)"},
                    "with_f64_state": {"value": e2e_value, "ms_per_step": e2e_ms / e2e_steps,
                                       "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": h2d,
                                       "state_finite": e2e_ok, "state_form": "float64 (x, v, F - I)",
                                       "what": "the float64 state (x, v, F - I) in mapped host buffers, read "
                                               "in place by pack, one step, written back by unpack"},
                    "with_memcpy": {"value": e2e_copy_value, "ms_per_step": e2e_copy_ms / e2e_steps,
                                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": h2d,
                                    "state_form": "float64 (x, v, F - I)",
                                    "what": "the float64 state in pinned host tensors, cudaMemcpyAsync to the "
                                            "device, pack, one step, unpack, cudaMemcpyAsync back"}},
            "gpu_launches": launches,
            "kernel_timing": {"events_every_nth_launch": TIMER_EVERY, "timed_launches": n_mom + n_def + n_str},
            "clocks": clk,
            "workloads": workloads,
        }
        if cb is not None:
            line["cpu_baseline"] = {k: cb[k] for k in ("value", "unit", "cores", "kind", "sample", "single_core")}
        print(json.dumps(line))
    ctx.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--e2e-steps", type=int, default=500)
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--profile", choices=["fp32", "fp64", "eu3d", "mlp", "relax", "comp"], default=None,
                    help="run only one workload (setup + warmup + steps) for ncu captures: the plate "
                         "(fp32 or fp64), the 3D Taylor-Green vortex of side --eu-n (eu3d, float32) or the "
                         "fused MLP forward over --mlp-rows rows (mlp), or float32 relaxation steps of the "
                         "8-sphere body at dp = 1/128 (relax)")
    ap.add_argument("--mlp-rows", type=int, default=262144, help="rows of the --profile mlp workload")
    ap.add_argument("--eu-n", type=int, default=64, help="lattice side of the --profile eu3d workload")
    ap.add_argument("--comp-nx", type=int, default=4096, help="strip length (particles) of the --profile comp workload")
    ap.add_argument("--no-tiles", action="store_true", help="--profile: without tile plans (per-pair geometry)")
    ap.add_argument("--kappa", type=float, default=1.6)
    ap.add_argument("--lanes", type=int, default=0, help="lanes per particle of the TL passes (0: tuned)")
    ap.add_argument("--headline-only", action="store_true", help="skip the other rows' workloads")
    ap.add_argument("--no-l2-persist", action="store_true",
                    help="launch the TL passes without their L2 access-policy windows (sph_set_l2_persist off)")
    ap.add_argument("--pipe", choices=["stream", "persistent", "bulk", "geom"], default=None,
                    help="how the planned TL passes get their pair entries (default: the context's)")
    ap.add_argument("--rows", default="", help="comma-separated names of the other rows to run (default: all)")
    ap.add_argument("--other-steps", type=int, default=100, help="timed steps of the other Eulerian workloads")
    ap.add_argument("--traffic", type=float, default=None,
                    help="ncu dram bytes per launch of the dominant kernel, if measured for the current kernels")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
