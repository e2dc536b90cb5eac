"""Seeded synthetic inputs shared by the CUDA path, the tests and the benchmark.

This module only lays particles out and fills initial fields; it holds none of
the SPH method's arithmetic (no kernel, neighbour, correction or update
formula).  Every random draw comes from ``numpy.random.default_rng(seed)``.

Workloads (all synthetic; the paper's experiments use analytic initial
conditions too):

* ``tgv2d``  periodic unit square, Taylor-Green vortex, lattice at (k+1/2) dp;
* ``tgv3d``  periodic cube of side 2 pi, 3D Taylor-Green vortex;
* ``plate``  0.2 x 0.02 x 0.2 m cantilever plate with a clamped root of four
  particle layers and the first bending mode as initial transverse velocity;
* ``sphere_body``  union of 8 seeded spheres filled with a jittered lattice;
* ``batched_tgv2d``  many 2D Taylor-Green cases of uneven size.

Each returns a dict; ``domain`` entries are plain dicts
``{dim, h, kappa, lo, len, periodic}`` that each side turns into its own type.
"""
import math

import numpy as np

H_FLUID = 1.3      # h / dp for fluids and relaxation (Sec. 4)
H_SOLID = 1.15     # h / dp for solids (Sec. 4)
KAPPA_TW = 1.6
KAPPA_SW = 2.0


def domain(dim, h, kappa, lo, length, periodic):
    return {"dim": int(dim), "h": float(h), "kappa": float(kappa),
            "lo": [float(x) for x in lo], "len": [float(x) for x in length],
            "periodic": [bool(p) for p in periodic]}


def lattice(counts, dp, lo=None):
    """Points (k + 1/2) dp + lo, x fastest; returns (dim, n) float64."""
    dim = len(counts)
    lo = np.zeros(dim) if lo is None else np.asarray(lo, dtype=np.float64)
    axes = [lo[k] + (np.arange(counts[k]) + 0.5) * dp for k in range(dim)]
    grids = np.meshgrid(*axes[::-1], indexing="ij")
    return np.stack([g.ravel() for g in grids[::-1]])


def tgv2d(nx=50, U=1.0, Re=100.0, rho0=1.0, c0_factor=10.0, kappa=KAPPA_TW):
    """2D Taylor-Green vortex on the periodic unit square.

    u = U sin(2 pi x) cos(2 pi y), v = -U cos(2 pi x) sin(2 pi y),
    p = (rho0 U^2 / 4)(cos 4 pi x + cos 4 pi y); velocity decays as
    exp(-8 pi^2 nu t) with nu = U L / Re, L = 1."""
    dp = 1.0 / nx
    h = H_FLUID * dp
    pos = lattice((nx, nx), dp)
    x, y = pos
    k = 2.0 * math.pi
    v = np.stack([U * np.sin(k * x) * np.cos(k * y), -U * np.cos(k * x) * np.sin(k * y)])
    p = 0.25 * rho0 * U * U * (np.cos(2 * k * x) + np.cos(2 * k * y))
    c0 = c0_factor * U
    mu = rho0 * U * 1.0 / Re
    dt = min(0.25 * h / (c0 + U), 0.125 * h * h * rho0 / mu)
    return {"pos": pos, "v": v, "p": p, "vol": np.full(pos.shape[1], dp * dp),
            "domain": domain(2, h, kappa, (0.0, 0.0), (1.0, 1.0), (True, True)),
            "dp": dp, "rho0": rho0, "c0": c0, "mu": mu, "U": U, "Re": Re, "dt": dt,
            "nu": mu / rho0, "decay_rate": 8.0 * math.pi ** 2 * mu / rho0}


def double_shear_layer(nx=128, rho=1.0 / 30.0, delta=0.05, rho0=1.0, c0_factor=10.0, kappa=KAPPA_TW):
    """The inviscid double periodic shear layer of Sec. 5 (unit square, mu = 0):
    u_x = tanh((y - 1/4)/rho) for y <= 1/2, tanh((3/4 - y)/rho) above; u_y = delta sin(2 pi x);
    rho = 1/30, delta = 0.05, uniform initial pressure.  c0 = 10 U with U = max|u| = 1,
    dt = 0.25 h/(c0 + U) (no viscous limit)."""
    dp = 1.0 / nx
    h = H_FLUID * dp
    pos = lattice((nx, nx), dp)
    x, y = pos
    ux = np.where(y <= 0.5, np.tanh((y - 0.25) / rho), np.tanh((0.75 - y) / rho))
    uy = delta * np.sin(2.0 * math.pi * x)
    U = 1.0
    c0 = c0_factor * U
    return {"pos": pos, "v": np.stack([ux, uy]), "p": np.zeros(pos.shape[1]),
            "vol": np.full(pos.shape[1], dp * dp),
            "domain": domain(2, h, kappa, (0.0, 0.0), (1.0, 1.0), (True, True)),
            "dp": dp, "rho0": rho0, "c0": c0, "mu": 0.0, "U": U, "dt": 0.25 * h / (c0 + U)}


def sod_strip(nx=400, ny=8, kappa=KAPPA_TW, gamma=1.4, cfl=0.2):
    """Two Sod shock tubes on a 2D strip periodic in x and y: (rho, p) = (1, 1) for
    x < 1/2 and (0.125, 0.1) for x >= 1/2, at rest, so that x = 1/2 is Sod's problem and
    x = 0 (= 1) its mirror image; the waves of the two stay apart until t ~ 0.15.
    Ideal gas gamma = 1.4; fixed dt = cfl h / 2.5 (2.5 bounds |u| + c of the solution)."""
    dp = 1.0 / nx
    h = H_FLUID * dp
    if ny * dp < 2.0 * kappa * h:
        raise ValueError("the strip must span two cut-offs: ny >= %g" % (2.0 * kappa * H_FLUID))
    pos = lattice((nx, ny), dp)
    left = pos[0] < 0.5
    rho = np.where(left, 1.0, 0.125)
    p = np.where(left, 1.0, 0.1)
    mom = np.zeros_like(pos)
    E = p / (gamma - 1.0)
    return {"pos": pos, "rho": rho, "mom": mom, "E": E, "vol": np.full(pos.shape[1], dp * dp),
            "domain": domain(2, h, kappa, (0.0, 0.0), (1.0, ny * dp), (True, True)),
            "dp": dp, "gamma": gamma, "dt": cfl * h / 2.5}


def tgv2d_exact_velocity(pos, U, nu, t):
    """Closed-form 2D Taylor-Green velocity at time t (incompressible solution)."""
    x, y = pos
    k = 2.0 * math.pi
    f = math.exp(-2.0 * k * k * nu * t)
    return np.stack([U * np.sin(k * x) * np.cos(k * y) * f, -U * np.cos(k * x) * np.sin(k * y) * f])


def tgv3d(n=128, Re=1600.0, rho0=1.0, c0=10.0, kappa=KAPPA_TW):
    """3D Taylor-Green vortex in the periodic cube [0, 2 pi)^3 (U = 1, L = 1)."""
    L = 2.0 * math.pi
    dp = L / n
    h = H_FLUID * dp
    pos = lattice((n, n, n), dp)
    x, y, z = pos
    v = np.stack([np.sin(x) * np.cos(y) * np.cos(z), -np.cos(x) * np.sin(y) * np.cos(z), np.zeros_like(x)])
    p = (rho0 / 16.0) * (np.cos(2 * x) + np.cos(2 * y)) * (np.cos(2 * z) + 2.0)
    mu = rho0 / Re
    U = 1.0
    dt = min(0.25 * h / (c0 + U), 0.125 * h * h * rho0 / mu)
    return {"pos": pos, "v": v, "p": p, "vol": np.full(pos.shape[1], dp ** 3),
            "domain": domain(3, h, kappa, (0.0, 0.0, 0.0), (L, L, L), (True, True, True)),
            "dp": dp, "rho0": rho0, "c0": c0, "mu": mu, "U": U, "Re": Re, "dt": dt}


def cantilever_mode(x, length, beta_l=1.875104068711961):
    """First Euler-Bernoulli bending mode of a clamped-free beam, normalised to 1 at the tip."""
    b = beta_l / length

    def f(s):
        k = (math.cosh(beta_l) + math.cos(beta_l)) / (math.sinh(beta_l) + math.sin(beta_l))
        return (np.cosh(b * s) - np.cos(b * s)) - k * (np.sinh(b * s) - np.sin(b * s))

    return f(np.maximum(x, 0.0)) / f(length)


def plate(dp=0.001, length=0.2, thickness=0.02, width=0.2, root_layers=4,
          rho0=1000.0, E=2.0e6, nu=0.3975, amp_factor=0.05, kappa=KAPPA_TW):
    """Oscillating cantilever plate (total-Lagrangian solid).

    Length along x in [0, length) plus a clamped root x in [-root_layers dp, 0);
    thickness along y, width along z.  Initial v_y = amp_factor c0 f(x)/f(L)."""
    nx = int(round(length / dp)) + root_layers
    ny = int(round(thickness / dp))
    nz = int(round(width / dp))
    lo = (-root_layers * dp, 0.0, 0.0)
    r0 = lattice((nx, ny, nz), dp, lo)
    fixed = (r0[0] < 0.0).astype(np.uint8)
    K = E / (3.0 * (1.0 - 2.0 * nu))
    c0 = math.sqrt(K / rho0)
    v = np.zeros_like(r0)
    v[1] = amp_factor * c0 * cantilever_mode(r0[0], length)
    v[:, fixed == 1] = 0.0
    h = H_SOLID * dp
    lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
    G = E / (2.0 * (1.0 + nu))
    vmax = amp_factor * c0
    dt = 0.5 * h / (c0 + vmax)
    margin = 2.0 * dp
    dom = domain(3, h, kappa, (lo[0] - margin, -margin, -margin),
                 (nx * dp + 2 * margin, ny * dp + 2 * margin, nz * dp + 2 * margin),
                 (False, False, False))
    return {"r0": r0, "v": v, "fixed": fixed, "vol": np.full(r0.shape[1], dp ** 3),
            "domain": dom, "dp": dp, "rho0": rho0, "E": E, "nu": nu, "lam": lam, "G": G,
            "c0": c0, "dt": dt}


def column(kind="twisting", n_side=10, side=1.0, height=6.0, root_layers=3, rho0=1100.0, E=17.0e6, nu=None,
           omega0=105.0, v0=10.0, kappa=KAPPA_TW):
    """The 3D columns of Sec. 5 (total-Lagrangian solids): a square section side x side in
    x-z (side / dp = n_side), height along y in [0, height), clamped below, y in
    [-root_layers dp, 0).
      twisting: nu = 0.499, rotation about the column axis with rate
                Omega(y) = omega0 sin(pi y / (2 height)): v = Omega(y) y_hat x (r - axis);
      bending:  nu = 0.45, uniform v = v0 (sqrt(3)/2, 1/2, 0).
    rho0 = 1100, E = 17 MPa, h = 1.15 dp, dt = 0.5 h/(c0 + v_max)."""
    if nu is None:
        nu = 0.499 if kind == "twisting" else 0.45
    dp = side / n_side
    ny = int(round(height / dp)) + root_layers
    lo = (0.0, -root_layers * dp, 0.0)
    r0 = lattice((n_side, ny, n_side), dp, lo)
    fixed = (r0[1] < 0.0).astype(np.uint8)
    v = np.zeros_like(r0)
    if kind == "twisting":
        rate = omega0 * np.sin(math.pi * r0[1] / (2.0 * height))
        dx, dz = r0[0] - 0.5 * side, r0[2] - 0.5 * side
        v[0] = rate * dz
        v[2] = -rate * dx
    elif kind == "bending":
        v[0] = v0 * math.sqrt(3.0) / 2.0
        v[1] = v0 * 0.5
    else:
        raise ValueError(kind)
    v[:, fixed == 1] = 0.0
    K = E / (3.0 * (1.0 - 2.0 * nu))
    c0 = math.sqrt(K / rho0)
    h = H_SOLID * dp
    lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
    G = E / (2.0 * (1.0 + nu))
    vmax = float(np.max(np.sqrt(np.sum(v * v, axis=0))))
    dt = 0.5 * h / (c0 + vmax)
    margin = 2.0 * dp
    dom = domain(3, h, kappa, (-margin, lo[1] - margin, -margin),
                 (side + 2 * margin, ny * dp + 2 * margin, side + 2 * margin), (False, False, False))
    return {"r0": r0, "v": v, "fixed": fixed, "vol": np.full(r0.shape[1], dp ** 3),
            "domain": dom, "dp": dp, "rho0": rho0, "E": E, "nu": nu, "lam": lam, "G": G,
            "c0": c0, "dt": dt}


def beam2d(dp=0.002, length=0.2, thickness=0.02, root_layers=4, periodic_x=False, rho0=1000.0, E=2.0e6,
           nu=0.3975, amp_factor=0.05, kappa=KAPPA_TW):
    """2D total-Lagrangian strip in x-y: the plate's section.

    Clamped root x in [-root_layers dp, 0) with the first-mode velocity of `plate`, or,
    with periodic_x, a strip periodic along x (no clamp) with v_y = amp c0 sin(2 pi x / L)."""
    nx = int(round(length / dp)) + (0 if periodic_x else root_layers)
    ny = int(round(thickness / dp))
    lo = (0.0 if periodic_x else -root_layers * dp, 0.0)
    r0 = lattice((nx, ny), dp, lo)
    fixed = np.zeros(r0.shape[1], dtype=np.uint8) if periodic_x else (r0[0] < 0.0).astype(np.uint8)
    K = E / (3.0 * (1.0 - 2.0 * nu))
    c0 = math.sqrt(K / rho0)
    v = np.zeros_like(r0)
    if periodic_x:
        v[1] = amp_factor * c0 * np.sin(2.0 * math.pi * r0[0] / (nx * dp))
    else:
        v[1] = amp_factor * c0 * cantilever_mode(r0[0], length)
        v[:, fixed == 1] = 0.0
    h = H_SOLID * dp
    lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
    G = E / (2.0 * (1.0 + nu))
    dt = 0.5 * h / (c0 + amp_factor * c0)
    margin = 2.0 * dp
    if periodic_x:
        dom = domain(2, h, kappa, (0.0, -margin), (nx * dp, ny * dp + 2 * margin), (True, False))
    else:
        dom = domain(2, h, kappa, (lo[0] - margin, -margin), (nx * dp + 2 * margin, ny * dp + 2 * margin),
                     (False, False))
    return {"r0": r0, "v": v, "fixed": fixed, "vol": np.full(r0.shape[1], dp ** 2), "domain": dom, "dp": dp,
            "rho0": rho0, "E": E, "nu": nu, "lam": lam, "G": G, "c0": c0, "dt": dt}


def sphere_union(seed, count=8, rmin=0.1, rmax=0.3):
    """Seeded centres U(0,1)^3 and radii U(rmin, rmax); rows (cx, cy, cz, r)."""
    rng = np.random.default_rng(seed)
    c = rng.uniform(0.0, 1.0, size=(count, 3))
    r = rng.uniform(rmin, rmax, size=count)
    return np.concatenate([c, r[:, None]], axis=1)


def sphere_body(seed, dp, jitter=0.25, count=8):
    """Lattice points (k + 1/2) dp inside the union of spheres, jittered by U(-j, j) dp."""
    spheres = sphere_union(seed, count)
    lo = np.min(spheres[:, :3] - spheres[:, 3:4], axis=0)
    hi = np.max(spheres[:, :3] + spheres[:, 3:4], axis=0)
    lo = np.floor(lo / dp) * dp
    counts = [int(math.ceil((hi[k] - lo[k]) / dp)) for k in range(3)]
    pts = lattice(counts, dp, lo)
    inside = np.zeros(pts.shape[1], dtype=bool)
    for s in spheres:
        inside |= np.sum((pts - s[:3, None]) ** 2, axis=0) <= s[3] * s[3]
    pts = pts[:, inside]
    rng = np.random.default_rng(seed + 7919)
    pts = pts + rng.uniform(-jitter, jitter, size=pts.shape) * dp
    h = H_FLUID * dp
    margin = 4.0 * dp
    dom = domain(3, h, 2.0, lo - margin, [counts[k] * dp + 2 * margin for k in range(3)],
                 (False, False, False))
    return {"pos": pts, "spheres": spheres, "vol": np.full(pts.shape[1], dp ** 3),
            "domain": dom, "dp": dp, "h": h}


def circle_body(dp, diameter=2.0, jitter=0.0, seed=0):
    """The geometry of the error analysis (Sec. 2.3.3): lattice points (k + 1/2) dp of
    the square [-D/2, D/2]^2 inside the circle of diameter D about the origin,
    optionally jittered by U(-j, j) dp; h = 1.3 dp, V = dp^2."""
    R = 0.5 * diameter
    m = int(math.ceil(diameter / dp - 1e-9))
    lo = -0.5 * m * dp
    pts = lattice([m, m], dp, [lo, lo])
    pts = pts[:, np.sum(pts * pts, axis=0) <= R * R]
    if jitter:
        rng = np.random.default_rng(seed + 104729)
        pts = pts + rng.uniform(-jitter, jitter, size=pts.shape) * dp
    h = H_FLUID * dp
    margin = 4.0 * dp
    dom = domain(2, h, 2.0, [lo - margin, lo - margin], [m * dp + 2 * margin] * 2, (False, False))
    return {"pos": np.ascontiguousarray(pts), "spheres": np.array([[0.0, 0.0, R]]), "vol": np.full(pts.shape[1], dp * dp),
            "domain": dom, "dp": dp, "h": h}


MLP_SHAPES = [(128, 128), (128,), (128, 128), (128,), (128, 128), (128,), (3, 128), (3,)]


def mlp_init(seed):
    """Seeded initial parameters of the 128-128-128-128-3 proposal network, flat float64:
    weights U(-a, a) with a = sqrt(6 / (fan_in + fan_out)), biases zero."""
    rng = np.random.default_rng(seed)
    parts = []
    for shape in MLP_SHAPES:
        if len(shape) == 2:
            a = math.sqrt(6.0 / (shape[0] + shape[1]))
            parts.append(rng.uniform(-a, a, size=shape).ravel())
        else:
            parts.append(np.zeros(shape))
    return np.concatenate(parts)


def batched_tgv2d(seed=0, ncases=64, nmin=64, nmax=1024, kappa=KAPPA_TW, scale=1.0):
    """Uneven batch of 2D Taylor-Green cases: n_c = round(exp U(ln nmin, ln nmax)) per side,
    Re in {100, 1000} by a fair coin.  ``scale`` shrinks every side (for small tests)."""
    rng = np.random.default_rng(seed)
    sides = np.rint(np.exp(rng.uniform(math.log(nmin), math.log(nmax), size=ncases))).astype(int)
    res = np.where(rng.uniform(size=ncases) < 0.5, 100.0, 1000.0)
    cases = []
    for nc, Re in zip(sides, res):
        nc = max(8, int(round(nc * scale)))
        cases.append(tgv2d(nx=nc, Re=float(Re), kappa=kappa))
    return cases
