"""The oracle's TL step on a process pool (the CPU baseline's all-core form) equals the
single-process oracle step bit for bit: the pool only splits the rows into blocks."""
import numpy as np

from oracle import kgc as OK
from oracle import neighbors as ON
from oracle import pool as OP
from oracle import tlsph as OT
from paper_2405_05155_gb300 import inputs


def test_pool_step_equals_the_oracle_step():
    c = inputs.plate(dp=0.01, kappa=1.6)
    d = c["domain"]
    dom = ON.Domain(d["dim"], d["h"], d["kappa"], d["lo"], d["len"], d["periodic"])
    rp, col = ON.neighbors_cells(c["r0"], dom)
    B0, _ = OK.kgc(c["r0"], c["vol"], rp, col, dom)
    prm = OT.TLParams(dom, c["dt"], c["rho0"], c["lam"], c["G"], OT.NEO_HOOKEAN)
    n = c["r0"].shape[1]
    x, v, F = c["r0"].copy(), c["v"].copy(), np.tile(np.eye(3), (n, 1, 1))
    xr, vr, Fr = x, v, F
    with OP.PoolStep(c["r0"], c["vol"], B0, c["fixed"], rp, col, prm, workers=2) as ps:
        assert len(ps.blocks) > 2 and ps.blocks[0][0] == 0 and ps.blocks[-1][1] == n
        for _ in range(3):
            x, v, F = ps.step(x, v, F)
            xr, vr, Fr = OT.step(c["r0"], c["vol"], B0, c["fixed"], xr, vr, Fr, rp, col, prm)
    assert np.array_equal(v, vr) and np.array_equal(F, Fr) and np.array_equal(x, xr)
    assert np.abs(v - c["v"]).max() > 0.0
