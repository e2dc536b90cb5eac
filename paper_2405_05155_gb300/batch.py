"""Batched Eulerian cases: per-case set-up through the C ABI (cell order, neighbour
lists, correction matrices, float32 packing, tile plan), then concatenation into the
sph_batch_state layout and stepping with sph_eulerian_step_batched.
"""
import ctypes

import torch

from . import _lib as L
from . import api


class EulerianBatch:
    def __init__(self, ctx, cases, integrator=api.SPH_TWO_PASS, tiles=True):
        self.ctx = ctx
        dev = ctx.device
        self.cases = cases
        self.sims = []
        self.orders = []
        recs, rps, cols = [], [], []
        off = 0
        nnz_off = 0
        self.table = (L.BatchCase * len(cases))()
        for c, case in enumerate(cases):
            d = case["domain"]
            pos = torch.tensor(case["pos"], dtype=torch.float64, device=dev)
            order = api.cell_order(ctx, d, pos)
            pos = pos[:, order].contiguous()
            oh = order.cpu().numpy()
            vol = torch.tensor(case["vol"][oh], dtype=torch.float64, device=dev)
            rp, col = api.build_neighbors(ctx, d, pos)
            B, _, _ = api.kgc(ctx, d, pos, vol, rp, col)
            drho = api.density_from_pressure(ctx, d, case["c0"], torch.tensor(case["p"], device=dev)[order])
            sim = api.Eulerian(ctx, d, pos, vol, B, rp, col, drho, case["v"][:, oh], case["dt"], case["rho0"],
                               case["c0"], case["mu"], precision=api.SPH_FP32_KAHAN, integrator=integrator,
                               tiles=tiles)
            n = pos.shape[1]
            t = self.table[c]
            t.offset, t.n, t.dim = off, n, d["dim"]
            t.periodic_mask = sum((1 << k) for k, p in enumerate(d["periodic"][: d["dim"]]) if p)
            t.h, t.dt, t.rho0, t.c0, t.mu, t.eta = d["h"], case["dt"], case["rho0"], case["c0"], case["mu"], 15.0
            for k in range(3):
                t.len[k] = d["len"][k] if k < d["dim"] else 1.0
            if sim.plan is not None:
                # the case's own tile plan (case-local indices); the batched step runs
                # its planned form when every case has one
                t.plan = sim.plan.data_ptr()
                t.plan_nnz, t.plan_maxm, t.plan_maxrow = sim.st.plan_nnz, sim.st.plan_maxm, sim.st.plan_maxrow
            recs.append(sim.rec)
            rps.append(rp[:-1] + nnz_off)
            cols.append(col + off)
            self.sims.append(sim)
            self.orders.append(order)
            off += n
            nnz_off += int(col.numel())
        rps.append(torch.tensor([nnz_off], dtype=torch.int64, device=dev))
        self.ntotal = off
        self.nnz = nnz_off
        self.row_ptr = torch.cat(rps).contiguous()
        self.col = torch.cat(cols).to(torch.int32).contiguous()
        self.rec = torch.cat(recs).contiguous()
        self.rec_tmp = self.rec.clone()
        self.st = L.BatchState()
        for name in ("row_ptr", "col", "rec", "rec_tmp"):
            setattr(self.st, name, getattr(self, name).data_ptr())

    def step(self, nsteps=1):
        L.check("sph_eulerian_step_batched", self.ctx.lib.sph_eulerian_step_batched(
            self.ctx.h, self.table, len(self.cases), ctypes.byref(self.st), int(nsteps), api._stream()), self.ctx.h)

    def autotune(self, trial_steps=5):
        lanes, block, ms = ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
        L.check("sph_autotune_batched", self.ctx.lib.sph_autotune_batched(
            self.ctx.h, self.table, len(self.cases), ctypes.byref(self.st), int(trial_steps), ctypes.byref(lanes),
            ctypes.byref(block), ctypes.byref(ms), api._stream()), self.ctx.h)
        return lanes.value, block.value, ms.value

    def fields(self, c):
        """(drho, v) float64 of case c (in its cell-sorted order), unpacked by sph_eulerian_unpack."""
        sim = self.sims[c]
        t = self.table[c]
        n = int(t.n)
        sim.rec.copy_(self.rec[16 * t.offset: 16 * (t.offset + n)])
        sim.unpack()
        return sim.drho, sim.v
