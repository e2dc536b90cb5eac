"""Total-Lagrangian SPH for solids, oracle version (test infrastructure).

Sec. 3.2.  Everything is taken in the reference configuration r0: neighbour lists,
kernel gradients grad0 W_ij and the correction matrices B0_i (Eq. 9 at r0).

* Eq. 28: rho = rho0 / J, rho0 dv/dt = div0 P^T, P = F S, J = det F.
* Eq. 29: St Venant-Kirchhoff S = lambda tr(E) I + 2 G E, with the Green strain
  E = (F^T F - I)/2 (implied).  The compressible neo-Hookean law
  S = G (I - C^-1) + lambda ln(J) C^-1, C = F^T F, is offered beside it.
* Eq. 30: rho0_i dv_i/dt = sum_j (P_i B0_i^T + P_j B0_j^T) grad0 W_ij V0_j.
* Eq. 31: dF_i/dt = (sum_j V0_j (v_j - v_i) (x) grad0 W_ij) B0_i; the printed
  "." between the velocity difference and the gradient is read as the dyadic
  product, the only reading that gives a matrix and makes the rate exact for
  linear velocity fields.

Readings for the time integration (the paper gives none): fixed dt; per step
stresses from F^n, a^n, v^{n+1} = v^n + dt a^n, then dF/dt with v^{n+1},
F^{n+1} = F^n + dt dF/dt and x^{n+1} = x^n + dt v^{n+1}.  Clamped (fixed)
particles keep v = 0 and F = I but stay in every neighbour sum.
"""
from dataclasses import dataclass

import numpy as np

from .kgc import kernel_gradients, sym_to_full
from .kernels import WENDLAND

SVK = 0
NEO_HOOKEAN = 1


@dataclass
class TLParams:
    dom: object          # neighbors.Domain of the reference configuration
    dt: float
    rho0: float
    lam: float
    G: float
    law: int = NEO_HOOKEAN


def lame(E, nu):
    """Lame parameter and shear modulus from Young's modulus and Poisson's ratio."""
    lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
    G = E / (2.0 * (1.0 + nu))
    return lam, G


def pk2_svk(F, lam, G):
    """Eq. 29: S = lambda tr(E) I + 2 G E, E = (F^T F - I)/2.  F: (n, d, d)."""
    d = F.shape[1]
    I = np.eye(d)
    C = np.einsum("nka,nkb->nab", F, F)
    E = 0.5 * (C - I)
    trE = np.trace(E, axis1=1, axis2=2)
    return lam * trE[:, None, None] * I + 2.0 * G * E


def pk2_neo_hookean(F, lam, G):
    """Compressible neo-Hookean: S = G (I - C^-1) + lambda ln(J) C^-1."""
    d = F.shape[1]
    I = np.eye(d)
    C = np.einsum("nka,nkb->nab", F, F)
    Cinv = np.linalg.inv(C)
    J = np.linalg.det(F)
    return G * (I - Cinv) + lam * np.log(J)[:, None, None] * Cinv


def first_piola(F, S):
    """P = F S (Sec. 3.2)."""
    return np.einsum("nab,nbc->nac", F, S)


def stress_matrix(F, B0s, prm):
    """M_i = P_i B0_i^T, the per-particle factor of Eq. 30."""
    dim = F.shape[1]
    S = pk2_neo_hookean(F, prm.lam, prm.G) if prm.law == NEO_HOOKEAN else pk2_svk(F, prm.lam, prm.G)
    P = first_piola(F, S)
    B0 = sym_to_full(B0s, dim)
    return np.einsum("nab,ncb->nac", P, B0)


def momentum_rate(r0, V0, M, row_ptr, col, dom, rho0):
    """Eq. 30 divided by rho0: dv_i/dt = (1/rho0) sum_j (M_i + M_j) grad0 W_ij V0_j."""
    n = r0.shape[1]
    dim = dom.dim
    i, j, rij, r, grad = kernel_gradients(r0, row_ptr, col, dom, WENDLAND)
    Msum = M[i] + M[j]                               # (m, d, d)
    f = np.einsum("mab,bm->am", Msum, grad) * V0[j]
    a = np.zeros((dim, n))
    for k in range(dim):
        a[k] = np.bincount(i, weights=f[k], minlength=n) / rho0
    return a


def deformation_rate(r0, V0, v, B0s, row_ptr, col, dom):
    """Eq. 31: dF_i/dt = (sum_j V0_j (v_j - v_i) (x) grad0 W_ij) B0_i, shape (n, d, d)."""
    n = r0.shape[1]
    dim = dom.dim
    i, j, rij, r, grad = kernel_gradients(r0, row_ptr, col, dom, WENDLAND)
    dv = v[:, j] - v[:, i]
    L = np.zeros((n, dim, dim))
    for a in range(dim):
        for b in range(dim):
            L[:, a, b] = np.bincount(i, weights=V0[j] * dv[a] * grad[b], minlength=n)
    B0 = sym_to_full(B0s, dim)
    return np.einsum("nab,nbc->nac", L, B0)


def step(r0, V0, B0s, fixed, x, v, F, row_ptr, col, prm):
    """One time step (stress, momentum, velocity, deformation rate, F, x)."""
    dom = prm.dom
    M = stress_matrix(F, B0s, prm)
    a = momentum_rate(r0, V0, M, row_ptr, col, dom, prm.rho0)
    free = fixed == 0
    v1 = np.where(free[None, :], v + prm.dt * a, 0.0)
    Fdot = deformation_rate(r0, V0, v1, B0s, row_ptr, col, dom)
    I = np.eye(dom.dim)
    F1 = np.where(free[:, None, None], F + prm.dt * Fdot, I[None, :, :])
    x1 = x + prm.dt * v1
    return x1, v1, F1


def run(r0, V0, B0s, fixed, x, v, F, row_ptr, col, prm, nsteps):
    for _ in range(nsteps):
        x, v, F = step(r0, V0, B0s, fixed, x, v, F, row_ptr, col, prm)
    return x, v, F


def energies(r0, V0, v, F, prm):
    """Kinetic and stored (strain) energy; the stored-energy density follows the law."""
    ke = 0.5 * prm.rho0 * np.sum(V0 * np.sum(v * v, axis=0))
    d = F.shape[1]
    C = np.einsum("nka,nkb->nab", F, F)
    if prm.law == NEO_HOOKEAN:
        J = np.linalg.det(F)
        lnJ = np.log(J)
        psi = 0.5 * prm.G * (np.trace(C, axis1=1, axis2=2) - d) - prm.G * lnJ + 0.5 * prm.lam * lnJ * lnJ
    else:
        E = 0.5 * (C - np.eye(d))
        trE = np.trace(E, axis1=1, axis2=2)
        psi = 0.5 * prm.lam * trE * trE + prm.G * np.einsum("nab,nab->n", E, E)
    return ke, float(np.sum(V0 * psi))


def time_step(h, E, nu, rho0, vmax):
    """Fixed step 0.5 h / (c0 + vmax) with c0 = sqrt(K/rho0), K = E / (3 (1 - 2 nu))."""
    K = E / (3.0 * (1.0 - 2.0 * nu))
    c0 = np.sqrt(K / rho0)
    return 0.5 * h / (c0 + vmax), float(c0)
