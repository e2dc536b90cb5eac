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


def _isnum(s):
    try:
        float(s)
        return True
    except ValueError:
        return False


# --------------------------------------------------------------------------- setup
def _setup_plate(api, inputs, ctx, kappa, dp=0.001):
    import torch
    c = inputs.plate(dp=dp, kappa=kappa)
    d = c["domain"]
    dev = ctx.device
    r0 = torch.tensor(c["r0"], dtype=torch.float64, device=dev)
    order = api.cell_order(ctx, d, r0)
    r0 = r0[:, order].contiguous()
    oh = order.cpu().numpy()
    vol = torch.tensor(c["vol"][oh], dtype=torch.float64, device=dev)
    rp, col = api.build_neighbors(ctx, d, r0)
    B0, fb, nfb = api.kgc(ctx, d, r0, vol, rp, col)
    return dict(c=c, d=d, r0=r0, vol=vol, rp=rp, col=col, B0=B0, v=c["v"][:, oh], fixed=c["fixed"][oh],
                nnz=int(col.numel()), n=int(r0.shape[1]), nfb=nfb)


def _solid(api, ctx, s, precision):
    c = s["c"]
    return api.TLSolid(ctx, s["d"], s["r0"], s["vol"], s["B0"], s["fixed"], s["rp"], s["col"], s["v"], c["dt"],
                       c["rho0"], c["lam"], c["G"], law=api.SPH_NEO_HOOKEAN, precision=precision)


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


def _max_over_ranks(x, world):
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _sum_over_ranks(x, world):
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def _alg_bytes_tl(n, nnz):
    """Algorithmic bytes of one float32 TL step, by pass (see the roofline notes in the design doc).

    momentum pass:  row_ptr 8 + geo 32 + own M 48 + v read/write 32 per particle, col 4 per pair;
    deformation pass: row_ptr 8 + geo 32 + v 16 + B0 24 + H read/write 72 + u read/write 24
                      + M write 48 per particle, col 4 per pair."""
    mom = n * (8 + 32 + 48 + 32) + 4 * nnz
    defo = n * (8 + 32 + 16 + 24 + 72 + 24 + 48) + 4 * nnz
    return mom, defo


def _cpu_baseline(steps_cap_s=12.0):
    """The oracle's TL step on a reduced plate (dp = 4 mm), timed on the host cores."""
    from oracle import kgc as OK
    from oracle import neighbors as ON
    from oracle import tlsph as OT
    from paper_2405_05155_gb300 import inputs
    c = inputs.plate(dp=0.004, kappa=1.6)
    d = c["domain"]
    dom = ON.Domain(d["dim"], d["h"], d["kappa"], d["lo"], d["len"], d["periodic"])
    rp, col = ON.neighbors_cells(c["r0"], dom)
    B0, _ = OK.kgc(c["r0"], c["vol"], rp, col, dom)
    prm = OT.TLParams(dom, c["dt"], c["rho0"], c["lam"], c["G"], OT.NEO_HOOKEAN)
    n = c["r0"].shape[1]
    x, v, F = c["r0"].copy(), c["v"].copy(), np.tile(np.eye(3), (n, 1, 1))
    steps = 0
    t0 = time.perf_counter()
    while time.perf_counter() - t0 < steps_cap_s or steps < 3:
        x, v, F = OT.step(c["r0"], c["vol"], B0, c["fixed"], x, v, F, rp, col, prm)
        steps += 1
    el = time.perf_counter() - t0
    pairs = 2 * col.size * steps
    return {"value": pairs / el, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": "float64 numpy oracle, plate at dp=0.004 m (%d particles, nnz=%d), %d time steps in %.1f s "
                      "(%.1f ms/step); single-threaded numpy" % (n, col.size, steps, el, 1e3 * el / steps),
            "ms_per_step": 1e3 * el / steps, "particles": n}


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
                             "sample": cb["sample"]},
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

    if args.profile:
        # profiling driver: the headline workload only (setup, then W + K float32 steps)
        s = _setup_plate(api, inputs, ctx, args.kappa)
        sol = _solid(api, ctx, s, api.SPH_FP64 if args.profile == "fp64" else api.SPH_FP32_KAHAN)
        sol.step(W + K)
        torch.cuda.synchronize()
        print(json.dumps({"profile": args.profile, "kappa": args.kappa, "particles": s["n"], "nnz": s["nnz"],
                          "steps": W + K}))
        ctx.close()
        return 0

    # headline: truncated kernel (1.6h), float32 + Kahan, per-kernel timing on
    s16 = _setup_plate(api, inputs, ctx, 1.6)
    sol = _solid(api, ctx, s16, api.SPH_FP32_KAHAN)
    sol.step(W)
    torch.cuda.synchronize()
    ctx.timing(True)
    clocks = ClockSampler(torch.cuda.current_device()) if rank == 0 else None
    ms, clk = _time_steps(ctx, sol, K, 0, world, clocks)
    t_mom, n_mom = ctx.timer(SPH_TIMER_TL_MOMENTUM)
    t_def, n_def = ctx.timer(SPH_TIMER_TL_DEFORM)
    t_str, n_str = ctx.timer(SPH_TIMER_TL_STRESS)
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
    ms20, _ = _time_steps(ctx, sol20, K, W, world)
    _, v20, H20 = sol20.fields()
    tw_vs_sw = {"v": rl2(v32, v20), "H": rl2(H32, H20)}
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
    traffic = args.traffic

    # end to end through the C ABI with host buffers: per step, copy the float64
    # state (x, v, F - I) from pinned host memory, pack, step, unpack, copy back
    e2e_steps = min(K, args.e2e_steps)
    sol_e = _solid(api, ctx, s16, api.SPH_FP32_KAHAN)
    hx = sol_e.x.cpu().pin_memory()
    hv = sol_e.v.cpu().pin_memory()
    hH = sol_e.H.cpu().pin_memory()
    h2d = (hx.numel() + hv.numel() + hH.numel()) * 8
    torch.cuda.synchronize()
    _barrier(world)
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record()
    for _ in range(e2e_steps):
        sol_e.x.copy_(hx, non_blocking=True)
        sol_e.v.copy_(hv, non_blocking=True)
        sol_e.H.copy_(hH, non_blocking=True)
        sol_e.pack()
        sol_e.step(1)
        sol_e.unpack()
        hx.copy_(sol_e.x, non_blocking=True)
        hv.copy_(sol_e.v, non_blocking=True)
        hH.copy_(sol_e.H, non_blocking=True)
    t1.record()
    torch.cuda.synchronize()
    e2e_ms = _max_over_ranks(t0.elapsed_time(t1), world)
    e2e_value = _sum_over_ranks(pairs_step * e2e_steps, world) / (e2e_ms * 1e-3)

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
                       "lanes_per_particle": ctx.get_lanes(api.SPH_PASS_TLSPH)},
            "kappa_2.0": {"ms_per_step": ms20 / K, "pair_interactions_per_s": 2 * s20["nnz"] * K / (ms20 * 1e-3),
                          "nnz": s20["nnz"]},
            "alpha_TW_over_SW": ms_step / (ms20 / K),
            "fp64": {"ms_per_step": ms64 / K, "pair_interactions_per_s": pairs_step * K / (ms64 * 1e-3)},
            "l2_fp32_vs_fp64": l2, "l2_tw_vs_sw": tw_vs_sw,
            "kernels_ms_avg": {"tl_momentum_pass": avg_mom, "tl_deformation_pass": avg_def,
                               "tl_stress_initial": t_str / max(n_str, 1)},
            "roofline": {"bound": "hbm", "kernel": dominant[0], "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic, "peak_source": peak_src,
                         "algorithmic_bytes_per_launch": dominant[1]},
            "e2e": {"value": e2e_value, "unit": UNIT, "steps": e2e_steps,
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": h2d,
                    "what": "per step: float64 (x, v, F-I) pinned host -> device, pack, one step, unpack, "
                            "device -> pinned host, through the C ABI"},
            "gpu_launches": n_mom + n_def + n_str,
            "clocks": clk,
        }
        if cb is not None:
            line["cpu_baseline"] = {k: cb[k] for k in ("value", "unit", "cores", "kind", "sample")}
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
    ap.add_argument("--profile", choices=["fp32", "fp64"], default=None,
                    help="run only the plate workload (setup + warmup + steps) for ncu captures")
    ap.add_argument("--kappa", type=float, default=1.6)
    ap.add_argument("--traffic", type=float, default=None,
                    help="ncu dram bytes per launch of the dominant kernel, if measured for this build")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
