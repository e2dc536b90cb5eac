"""The oracle's total-Lagrangian step on several host cores (test infrastructure).

This is the plain float64 oracle of ``oracle.tlsph``, unchanged, with its two pair sums
(Eq. 30, Eq. 31) evaluated over blocks of rows by a pool of worker processes.  A block
[lo, hi) is handed to ``momentum_rate`` / ``deformation_rate`` as a small particle set:
the block's rows followed by their neighbours outside the block (gathered copies of the
same float64 values), with the block's CSR rows renumbered into it and empty rows for the
neighbours.  The oracle code then computes the block's rows with the same operations in
the same order as over the whole list, and they are copied into place: every row's value
comes from one call of the oracle's own code, and a step of ``PoolStep`` equals
``tlsph.step`` bit for bit (tested).

The per-particle stress factor M_i is computed on the same blocks.  Only tests and
bench.py's CPU-baseline leg use this module.  Workers are started with the ``spawn``
method: they never inherit a parent's CUDA context.  Arrays that change every step (F, M,
v) and the block results go through shared memory.
"""
import multiprocessing as mp
import os
from multiprocessing import shared_memory

import numpy as np

from . import tlsph as OT

_W = {}


def host_cores():
    """Cores this process may run on."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def _attach(name, shape):
    shm = shared_memory.SharedMemory(name=name)
    return shm, np.ndarray(shape, dtype=np.float64, buffer=shm.buf)


def _init(static, names):
    _W.clear()
    _W.update(static)
    n, dim = static["n"], static["dom"].dim
    _W["shm"] = []
    for key, shape in (("M", (n, dim, dim)), ("v", (dim, n)), ("a", (dim, n)), ("Fd", (n, dim, dim)),
                       ("F", (n, dim, dim))):
        shm, arr = _attach(names[key], shape)
        _W["shm"].append(shm)
        _W[key] = arr


def block_set(row_ptr, col, lo, hi):
    """Particle set of the row block [lo, hi): global indices (the rows, then the other
    neighbours in ascending order) and the block's CSR in those local indices."""
    p0, p1 = row_ptr[lo], row_ptr[hi]
    cj = col[p0:p1].astype(np.int64)
    halo = np.setdiff1d(np.unique(cj), np.arange(lo, hi))
    idx = np.concatenate([np.arange(lo, hi), halo])
    order = np.argsort(idx)
    loc_col = order[np.searchsorted(idx[order], cj)]
    rp = np.concatenate([row_ptr[lo:hi + 1] - p0, np.full(halo.size, p1 - p0)])
    return idx, rp, loc_col.astype(col.dtype)


def _task(args):
    kind, b = args
    lo, hi, idx, rp, col = _W["blocks"][b]
    cache = _W.setdefault("cache", {})
    if b not in cache:
        cache[b] = (_W["r0"][:, idx], _W["V0"][idx], _W["B0s"][:, idx])
    r0, V0, B0s = cache[b]
    if kind == 2:
        # the stress factor is per particle: the block's rows alone
        _W["M"][lo:hi] = OT.stress_matrix(_W["F"][lo:hi], _W["B0s"][:, lo:hi], _W["prm"])
    elif kind == 0:
        a = OT.momentum_rate(r0, V0, _W["M"][idx], rp, col, _W["dom"], _W["rho0"])
        _W["a"][:, lo:hi] = a[:, :hi - lo]
    else:
        Fd = OT.deformation_rate(r0, V0, _W["v"][:, idx], B0s, rp, col, _W["dom"])
        _W["Fd"][lo:hi] = Fd[:hi - lo]
    return hi - lo


class PoolStep:
    """tlsph.step with the pair sums on `workers` processes (blocks of about equal pair counts)."""

    def __init__(self, r0, V0, B0s, fixed, row_ptr, col, prm, workers=None):
        self.r0, self.V0, self.B0s, self.fixed = r0, V0, B0s, fixed
        self.row_ptr, self.col, self.prm = row_ptr, col, prm
        n, dim = r0.shape[1], prm.dom.dim
        self.n, self.workers = n, max(1, int(workers or host_cores()))
        shapes = {"M": (n, dim, dim), "v": (dim, n), "a": (dim, n), "Fd": (n, dim, dim), "F": (n, dim, dim)}
        self._shm = {k: shared_memory.SharedMemory(create=True, size=max(8, int(np.prod(s)) * 8))
                     for k, s in shapes.items()}
        self.arr = {k: np.ndarray(shapes[k], dtype=np.float64, buffer=self._shm[k].buf) for k in shapes}
        # blocks of about equal pair counts, two per worker
        nb = 2 * self.workers
        cuts = np.searchsorted(row_ptr, np.linspace(0, row_ptr[-1], nb + 1)[1:-1])
        edges = np.unique(np.concatenate([[0], np.clip(cuts, 0, n), [n]]))
        self.blocks = [(int(edges[k]), int(edges[k + 1])) for k in range(len(edges) - 1)]
        sets = [(lo, hi) + block_set(row_ptr, col, lo, hi) for lo, hi in self.blocks]
        static = {"r0": r0, "V0": V0, "B0s": B0s, "blocks": sets, "dom": prm.dom, "rho0": prm.rho0, "n": n,
                  "prm": prm}
        names = {k: s.name for k, s in self._shm.items()}
        self.pool = mp.get_context("spawn").Pool(self.workers, initializer=_init, initargs=(static, names))

    def step(self, x, v, F):
        """One time step, as tlsph.step."""
        prm = self.prm
        self.arr["F"][...] = F
        self.pool.map(_task, [(2, b) for b in range(len(self.blocks))])
        self.pool.map(_task, [(0, b) for b in range(len(self.blocks))])
        a = self.arr["a"].copy()
        free = self.fixed == 0
        v1 = np.where(free[None, :], v + prm.dt * a, 0.0)
        self.arr["v"][...] = v1
        self.pool.map(_task, [(1, b) for b in range(len(self.blocks))])
        Fdot = self.arr["Fd"].copy()
        I = np.eye(prm.dom.dim)
        F1 = np.where(free[:, None, None], F + prm.dt * Fdot, I[None, :, :])
        x1 = x + prm.dt * v1
        return x1, v1, F1

    def close(self):
        if self.pool is not None:
            self.pool.close()
            self.pool.join()
            self.pool = None
        for s in self._shm.values():
            s.close()
            s.unlink()
        self._shm = {}

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
