"""Seeded synthetic inputs shared by the oracle-side tests and the CUDA path.

This module holds no arithmetic of the method itself: it describes meshes
(`MeshSpec`), derives cell-centre coordinates from a block list, and writes
initial conditions.  Both sides receive the same block list (level and integer
block coordinates per leaf), so the same initial state reaches both.

Workloads follow the shapes of the paper's Euler benchmarks (Sec. 4-5) with
synthetic initial data:
  * Kelvin-Helmholtz band in 2D (`kelvin_helmholtz`),
  * a random smooth 3D density/velocity field (`fourier3d`),
  * a spherical over-pressure region (`over_pressure`),
  * Sod shock tubes (`shock_tube`), a smooth density wave (`density_wave`),
  * the linear field phi = x + 2y + 3z of the AMR ghost-cell test (Sec. 4.3),
  * the advected scalar of Sec. 4.1: the smoothed sphere (Eq. 17), the
    Gaussian (Eq. 19) and a smooth periodic wave, with exact solutions.
Random numbers come from numpy's PCG64 (mode parameters) or from SplitMix64
(per-cell noise), so that a cell's noise depends only on its global index.
"""
from __future__ import annotations

import dataclasses
from typing import Sequence

import numpy as np

BC_PERIODIC, BC_DIRICHLET, BC_NEUMANN, BC_DATA = 0, 1, 2, 3


@dataclasses.dataclass
class MeshSpec:
    """Problem statement shared by both sides (Sec. 2.2-2.4).

    ntrees: brick of trees per dimension; periodic: per dimension;
    bc_type/bc_val: per face direction -x,+x,-y,+y,-z,+z and variable.
    """

    ndim: int = 2
    N: int = 16
    ng: int = 2
    ntrees: Sequence[int] = (16, 16, 1)
    periodic: Sequence[int] = (1, 1, 1)
    lo: Sequence[float] = (0.0, 0.0, 0.0)
    length: Sequence[float] = (1.0, 1.0, 1.0)
    max_level: int = 0
    gamma: float = 1.4
    cfl: float = 0.5
    bc_type: Sequence[int] = (0, 0, 0, 0, 0, 0)
    bc_val: Sequence[Sequence[float]] = tuple(tuple(0.0 for _ in range(8)) for _ in range(6))
    limiter: int = 0          # 0 minmod, 1 MC, 2 van Leer (MUSCL slopes), 3 WENO5 (ng >= 3),
                              # 4 Koren, 5 WENO3, 6 first-order upwind
    flux: int = 0             # 0 Rusanov, 1 HLL
    gravity: Sequence[float] = (0.0, 0.0, 0.0)   # source term S = (0, rho g, rho g.u)
    diagonal_ghosts: int = 0  # 1: also fill edge/corner ghosts held by same-level leaves
    physics: int = 0          # 0 Euler gas dynamics, 1 scalar advection (one variable)
    velocity: Sequence[float] = (0.0, 0.0, 0.0)   # uniform advection velocity

    @property
    def nvar(self) -> int:
        return 1 if self.physics == 1 else self.ndim + 2

    @property
    def side(self) -> int:
        return self.N + 2 * self.ng

    @property
    def ncell(self) -> int:
        return self.side ** self.ndim

    def block_shape(self):
        return (self.nvar,) + (self.side,) * self.ndim

    def tree_size(self, d: int) -> float:
        return self.length[d] / self.ntrees[d]

    def dx(self, d: int, lev) -> np.ndarray:
        return self.length[d] / self.ntrees[d] / (self.N * np.power(2.0, lev))


def block_geometry(spec: MeshSpec, lev: np.ndarray, g: np.ndarray):
    """Origins [nb,3] and cell sizes [nb,3] of the blocks (lev [nb], g [nb,3])."""
    lev = np.asarray(lev, dtype=np.int64)
    g = np.asarray(g, dtype=np.int64).reshape(-1, 3)
    origin = np.zeros((len(lev), 3))
    dx = np.ones((len(lev), 3))
    for d in range(spec.ndim):
        size = spec.tree_size(d) / np.power(2.0, lev)
        origin[:, d] = spec.lo[d] + g[:, d] * size
        dx[:, d] = size / spec.N
    return origin, dx


def cell_centres(spec: MeshSpec, lev, g, with_ghosts=True):
    """Coordinate arrays X[d] with shape [nb] + [side]*ndim (k, j, i order)."""
    origin, dx = block_geometry(spec, lev, g)
    nb = origin.shape[0]
    n = spec.side if with_ghosts else spec.N
    off = -spec.ng if with_ghosts else 0
    idx = np.arange(n) + off + 0.5
    out = []
    for d in range(spec.ndim):
        c = origin[:, d, None] + idx[None, :] * dx[:, d, None]
        shape = [nb] + [1] * spec.ndim
        shape[spec.ndim - d] = n          # axis order: block, (k), j, i
        out.append(np.broadcast_to(c.reshape(shape), [nb] + [n] * spec.ndim))
    return out


def global_cell_ids(spec: MeshSpec, lev, g):
    """Global index of every interior cell at its own level (x fastest)."""
    lev = np.asarray(lev, dtype=np.int64)
    g = np.asarray(g, dtype=np.int64).reshape(-1, 3)
    nb = len(lev)
    n = spec.N
    side = spec.side
    ids = np.zeros([nb] + [side] * spec.ndim, dtype=np.uint64)
    loc = np.arange(side, dtype=np.int64) - spec.ng
    ext = [spec.ntrees[d] * n * (1 << lev) for d in range(spec.ndim)]
    gx = g[:, 0, None] * n + loc[None, :]
    gy = g[:, 1, None] * n + loc[None, :]
    if spec.ndim == 2:
        ids = gx[:, None, :] + ext[0][:, None, None] * gy[:, :, None]
    else:
        gz = g[:, 2, None] * n + loc[None, :]
        ids = (gx[:, None, None, :] + ext[0][:, None, None, None] *
               (gy[:, None, :, None] + ext[1][:, None, None, None] * gz[:, :, None, None]))
    return np.asarray(ids, dtype=np.int64)


def splitmix64(x: np.ndarray) -> np.ndarray:
    """SplitMix64 output for counter x (uint64 array)."""
    with np.errstate(over="ignore"):
        z = (x.astype(np.uint64) + np.uint64(0x9E3779B97F4A7C15))
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def uniform_from_counter(seed: int, ids: np.ndarray) -> np.ndarray:
    """U(-1, 1) from SplitMix64(seed xor id), 53-bit resolution."""
    z = splitmix64(np.uint64(seed) ^ ids.astype(np.uint64))
    return (z >> np.uint64(11)).astype(np.float64) * (2.0 / 9007199254740992.0) - 1.0


def primitive_to_state(spec: MeshSpec, rho, vel, p):
    """Conservative block array [nb, V, side^d] from primitive fields."""
    gam = spec.gamma
    nb = rho.shape[0]
    u = np.zeros((nb, spec.nvar) + rho.shape[1:])
    u[:, 0] = rho
    ke = np.zeros_like(rho)
    for d in range(spec.ndim):
        u[:, 1 + d] = rho * vel[d]
        ke = ke + vel[d] * vel[d]
    u[:, spec.ndim + 1] = p / (gam - 1.0) + 0.5 * rho * ke
    return u.reshape(nb, spec.nvar, -1).copy()


def mask_interior(spec: MeshSpec, u: np.ndarray) -> np.ndarray:
    """Zero every non-interior cell (ghosts are the method's job to fill)."""
    nb = u.shape[0]
    v = u.reshape((nb, spec.nvar) + (spec.side,) * spec.ndim)
    m = np.zeros((spec.side,) * spec.ndim, dtype=bool)
    sl = tuple(slice(spec.ng, spec.ng + spec.N) for _ in range(spec.ndim))
    m[sl] = True
    v[:, :, ~m] = 0.0
    return u


def kelvin_helmholtz(spec: MeshSpec, lev, g, seed=0):
    """KH band: rho=2 and vx=+0.5 for |y-0.5|<0.25, rho=1 and vx=-0.5 elsewhere,
    p=2.5, vy = 0.01 sin(4 pi x) + U(-1e-3, 1e-3) per cell."""
    X = cell_centres(spec, lev, g)
    inside = np.abs(X[1] - 0.5) < 0.25
    rho = np.where(inside, 2.0, 1.0)
    vx = np.where(inside, 0.5, -0.5)
    noise = 1e-3 * uniform_from_counter(seed, global_cell_ids(spec, lev, g))
    vy = 0.01 * np.sin(4.0 * np.pi * X[0]) + noise
    p = np.full_like(rho, 2.5)
    vel = [vx, vy] + ([np.zeros_like(rho)] if spec.ndim == 3 else [])
    return mask_interior(spec, primitive_to_state(spec, rho, vel, p))


def fourier_modes(seed: int, nmodes=8, kmax=4):
    rng = np.random.Generator(np.random.PCG64(seed))
    ks, amps, phases = [], [], []
    while len(ks) < nmodes:
        k = rng.integers(-kmax, kmax + 1, size=3)
        if not np.any(k):
            continue
        ks.append(k)
        amps.append(rng.uniform(0.5, 1.0))
        phases.append(rng.uniform(0.0, 2.0 * np.pi))
    return np.array(ks), np.array(amps), np.array(phases)


def _fourier_sum(X, ndim, ks, amps, phases):
    s = np.zeros_like(X[0])
    for k, a, ph in zip(ks, amps, phases):
        arg = ph + sum(2.0 * np.pi * k[d] * X[d] for d in range(ndim))
        s = s + a * np.sin(arg)
    return s / np.sum(amps)


def fourier3d(spec: MeshSpec, lev, g, seed=1):
    """rho = 1 + 0.5 S, S a normalised sum of 8 seeded Fourier modes (|S| < 1);
    p = 1; each velocity component 0.1 times its own seeded mode sum."""
    X = cell_centres(spec, lev, g)
    rho = 1.0 + 0.5 * _fourier_sum(X, spec.ndim, *fourier_modes(seed))
    vel = [0.1 * _fourier_sum(X, spec.ndim, *fourier_modes(seed * 7919 + 1 + d)) for d in range(spec.ndim)]
    p = np.ones_like(rho)
    return mask_interior(spec, primitive_to_state(spec, rho, vel, p))


def over_pressure(spec: MeshSpec, lev, g, centre, radius=0.1, p_in=100.0, p_out=1.0):
    """rho = 1, v = 0, p = p_in inside the sphere, p_out outside."""
    X = cell_centres(spec, lev, g)
    r2 = sum((X[d] - centre[d]) ** 2 for d in range(spec.ndim))
    p = np.where(r2 < radius * radius, p_in, p_out)
    rho = np.ones_like(p)
    vel = [np.zeros_like(p) for _ in range(spec.ndim)]
    return mask_interior(spec, primitive_to_state(spec, rho, vel, p))


def shock_tube(spec: MeshSpec, lev, g, x0=0.5, axis=0, left=(1.0, 0.0, 1.0), right=(0.125, 0.0, 0.1)):
    """Riemann problem along `axis`: (rho, v_axis, p) = left for x < x0, right after."""
    X = cell_centres(spec, lev, g)
    L = X[axis] < x0
    rho = np.where(L, left[0], right[0])
    vn = np.where(L, left[1], right[1])
    p = np.where(L, left[2], right[2])
    vel = [vn if d == axis else np.zeros_like(rho) for d in range(spec.ndim)]
    return mask_interior(spec, primitive_to_state(spec, rho, vel, p))


def density_wave(spec: MeshSpec, lev, g, amp=0.2, vel=(1.0, 1.0, 1.0)):
    """rho = 1 + amp sin(2 pi sum_d x_d), uniform velocity, p = 1 (an exact
    translating solution of the Euler equations)."""
    X = cell_centres(spec, lev, g)
    s = sum(X[d] for d in range(spec.ndim))
    rho = 1.0 + amp * np.sin(2.0 * np.pi * s)
    v = [np.full_like(rho, vel[d]) for d in range(spec.ndim)]
    return mask_interior(spec, primitive_to_state(spec, rho, v, np.ones_like(rho)))


def density_wave_exact(spec: MeshSpec, lev, g, t, amp=0.2, vel=(1.0, 1.0, 1.0)):
    X = cell_centres(spec, lev, g)
    s = sum(X[d] - vel[d] * t for d in range(spec.ndim))
    return 1.0 + amp * np.sin(2.0 * np.pi * s)


def linear_field(spec: MeshSpec, lev, g, with_ghosts=False):
    """phi = x + 2y + 3z (Sec. 4.3), variable v holds (v+1) phi."""
    X = cell_centres(spec, lev, g)
    coef = (1.0, 2.0, 3.0)
    phi = sum(coef[d] * X[d] for d in range(spec.ndim))
    nb = phi.shape[0]
    u = np.stack([(v + 1.0) * phi for v in range(spec.nvar)], axis=1).reshape(nb, spec.nvar, -1).copy()
    return u if with_ghosts else mask_interior(spec, u)


def linear_face_values(spec: MeshSpec, lev, g, bc_entries):
    """bc_data for Dirichlet faces of the linear field: one row per boundary
    entry (face, dst) in the given order, values at face centres
    [n_bf, V, N^(d-1)] (lower tangential dimension fastest)."""
    origin, dx = block_geometry(spec, lev, g)
    coef = (1.0, 2.0, 3.0)
    n = spec.N
    nface = n ** (spec.ndim - 1)
    out = np.zeros((len(bc_entries), spec.nvar, nface))
    for r, (face, dst) in enumerate(bc_entries):
        nd, side = face // 2, face % 2
        td = [d for d in range(spec.ndim) if d != nd]
        xn = origin[dst, nd] + (n * dx[dst, nd] if side else 0.0)
        t = np.arange(n) + 0.5
        if spec.ndim == 2:
            xt0 = origin[dst, td[0]] + t * dx[dst, td[0]]
            phi = coef[nd] * xn + coef[td[0]] * xt0
        else:
            xt0 = origin[dst, td[0]] + t[None, :] * dx[dst, td[0]]
            xt1 = origin[dst, td[1]] + t[:, None] * dx[dst, td[1]]
            phi = (coef[nd] * xn + coef[td[0]] * xt0 + coef[td[1]] * xt1).reshape(-1)
        for v in range(spec.nvar):
            out[r, v] = (v + 1.0) * np.asarray(phi).reshape(-1)
    return out


def ball_flags(spec: MeshSpec, lev, g, centre, radius_per_level):
    """+1 for blocks at level l < len(radius_per_level) whose box meets the
    ball of radius radius_per_level[l] around `centre` (periodic images
    ignored); 0 elsewhere."""
    origin, dx = block_geometry(spec, lev, g)
    lev = np.asarray(lev)
    flags = np.zeros(len(lev), dtype=np.int8)
    for b in range(len(lev)):
        if lev[b] >= len(radius_per_level):
            continue
        r = radius_per_level[lev[b]]
        d2 = 0.0
        for d in range(spec.ndim):
            lo = origin[b, d]
            hi = lo + spec.N * dx[b, d]
            c = min(max(centre[d], lo), hi)
            d2 += (c - centre[d]) ** 2
        if d2 <= r * r:
            flags[b] = 1
    return flags


def point_flags(spec: MeshSpec, lev, g, point, max_level):
    """+1 for blocks below max_level whose box contains `point` (Sec. 4.3)."""
    origin, dx = block_geometry(spec, lev, g)
    lev = np.asarray(lev)
    flags = np.zeros(len(lev), dtype=np.int8)
    for b in range(len(lev)):
        if lev[b] >= max_level:
            continue
        inside = all(origin[b, d] <= point[d] <= origin[b, d] + spec.N * dx[b, d] for d in range(spec.ndim))
        if inside:
            flags[b] = 1
    return flags


def normal_shock_state(mach, gamma=1.4, rho1=1.0, p1=1.0):
    """Post-shock (rho, u, p) of a normal shock of Mach number `mach` moving
    into gas at rest (rho1, p1), from the Rankine-Hugoniot jump conditions:
    rho2/rho1 = (g+1) M^2 / ((g-1) M^2 + 2), p2/p1 = (2 g M^2 - (g-1)) / (g+1),
    u2 = M c1 (1 - rho1 / rho2)."""
    m2 = mach * mach
    rho2 = rho1 * (gamma + 1.0) * m2 / ((gamma - 1.0) * m2 + 2.0)
    p2 = p1 * (2.0 * gamma * m2 - (gamma - 1.0)) / (gamma + 1.0)
    c1 = np.sqrt(gamma * p1 / rho1)
    return rho2, mach * c1 * (1.0 - rho1 / rho2), p2


def sphere_and_shock(spec: MeshSpec, lev, g, centre, radius=0.1, p_in=100.0, shock_x=0.1, mach=3.0):
    """Over-pressure sphere (rho = 1, p = p_in inside, 1 outside) and a planar
    shock of Mach `mach` at x = shock_x moving in +x (post-shock state behind)."""
    X = cell_centres(spec, lev, g)
    r2 = sum((X[d] - centre[d]) ** 2 for d in range(spec.ndim))
    rho2, u2, p2 = normal_shock_state(mach, spec.gamma)
    behind = X[0] < shock_x
    rho = np.where(behind, rho2, 1.0)
    p = np.where(behind, p2, np.where(r2 < radius * radius, p_in, 1.0))
    vel = [np.where(behind, u2, 0.0)] + [np.zeros_like(rho) for _ in range(spec.ndim - 1)]
    return mask_interior(spec, primitive_to_state(spec, rho, vel, p))


def rayleigh_taylor(spec: MeshSpec, lev, g, h0=0.8, rho_hi=1.0, rho_lo=0.1, delta=0.05, p_top=1.0):
    """Rayleigh-Taylor state of Sec. 4.2: heavy fluid (rho_hi) above the
    interface h = h0 + delta sin(2 pi x) [sin(2 pi y) in 3D], light fluid
    below, at rest, pressure in hydrostatic balance with g = -1 along the last
    dimension (p = p_top at the top); cell-centre sampling."""
    X = cell_centres(spec, lev, g)
    vert = X[spec.ndim - 1]
    if spec.ndim == 3:
        h = h0 + delta * np.sin(2.0 * np.pi * X[0]) * np.sin(2.0 * np.pi * X[1])
    else:
        h = h0 + delta * np.sin(2.0 * np.pi * X[0])
    top = spec.lo[spec.ndim - 1] + spec.length[spec.ndim - 1]
    heavy = vert > h
    rho = np.where(heavy, rho_hi, rho_lo)
    p = np.where(heavy, p_top + rho_hi * (top - vert), p_top + rho_hi * (top - h) + rho_lo * (h - vert))
    vel = [np.zeros_like(rho) for _ in range(spec.ndim)]
    return mask_interior(spec, primitive_to_state(spec, rho, vel, p))


def rayleigh_taylor_spec(ndim=3, N=16, ntrees=None, limiter=2, rho_hi=1.0, rho_lo=0.1, ng=None, **kw) -> MeshSpec:
    """Sec. 4.2 setup: unit square/cube, periodic horizontally, gamma = 5/3,
    g = -1 along the last dimension; the vertical faces are Neumann with the
    hydrostatic gradient of the energy (outward derivative of E = outward
    dp/dn / (gamma - 1): rho_lo / (gamma - 1) at the bottom, -rho_hi /
    (gamma - 1) at the top) and zero gradient for the other variables."""
    gam = 5.0 / 3.0
    nt = ntrees if ntrees is not None else tuple([256 // N] * ndim + [1] * (3 - ndim))
    V = ndim + 2
    per = [1, 1, 1]
    per[ndim - 1] = 0
    bct = [0] * 6
    bct[2 * (ndim - 1)] = bct[2 * (ndim - 1) + 1] = BC_NEUMANN
    bcv = [[0.0] * 8 for _ in range(6)]
    bcv[2 * (ndim - 1)][V - 1] = rho_lo / (gam - 1.0)
    bcv[2 * (ndim - 1) + 1][V - 1] = -rho_hi / (gam - 1.0)
    grav = [0.0, 0.0, 0.0]
    grav[ndim - 1] = -1.0
    if ng is None:
        ng = 3 if limiter == 3 else 2
    return MeshSpec(ndim=ndim, N=N, ng=ng, ntrees=tuple(nt), periodic=tuple(per), gamma=gam, cfl=0.5,
                    bc_type=tuple(bct), bc_val=tuple(tuple(r) for r in bcv), limiter=limiter,
                    gravity=tuple(grav), **kw)


# ------------------------------------------------------ scalar advection --

def advection_spec(ndim=2, N=16, ntrees=None, limiter=2, velocity=(1.0, 1.0, 1.0), ng=None, **kw) -> MeshSpec:
    """Sec. 4.1 setup: the scalar advection equation (Eq. 13) on the periodic
    unit square/cube with a uniform velocity (default v_i = 1)."""
    nt = ntrees if ntrees is not None else tuple([4] * ndim + [1] * (3 - ndim))
    if ng is None:
        ng = 3 if limiter == 3 else 2
    vel = tuple(float(velocity[d]) if d < ndim else 0.0 for d in range(3))
    return MeshSpec(ndim=ndim, N=N, ng=ng, ntrees=tuple(nt), periodic=(1, 1, 1), limiter=limiter,
                    physics=1, velocity=vel, **kw)


def _periodic_distance(spec: MeshSpec, X, centre):
    """Distance to `centre` under the minimum-image convention of the
    periodic domain."""
    d2 = 0.0
    for d in range(spec.ndim):
        L = spec.length[d]
        r = X[d] - centre[d]
        r = r - L * np.round(r / L)
        d2 = d2 + r * r
    return np.sqrt(d2)


def _moved_centre(spec: MeshSpec, t):
    return [spec.lo[d] + 0.5 * spec.length[d] + spec.velocity[d] * t for d in range(spec.ndim)]


def advection_sphere(spec: MeshSpec, lev, g, t=0.0, R=0.1, delta=0.05):
    """Eq. 17: 1 inside d < R - delta, 1 - 3q^2 + 2q^3 with q = 1 + (d - R) /
    delta in the shell, 0 outside; d is the distance from the domain centre
    (moved by v t, periodic images), sampled at cell centres."""
    X = cell_centres(spec, lev, g)
    d = _periodic_distance(spec, X, _moved_centre(spec, t))
    q = 1.0 + (d - R) / delta
    rho = np.where(d < R - delta, 1.0, np.where(d < R, 1.0 - 3.0 * q * q + 2.0 * q * q * q, 0.0))
    return mask_interior(spec, rho.reshape(len(rho), 1, -1).copy())


def advection_gaussian(spec: MeshSpec, lev, g, t=0.0, R=0.1):
    """Eq. 19: exp(-d^2 / R^2) around the domain centre moved by v t."""
    X = cell_centres(spec, lev, g)
    d = _periodic_distance(spec, X, _moved_centre(spec, t))
    rho = np.exp(-(d * d) / (R * R))
    return mask_interior(spec, rho.reshape(len(rho), 1, -1).copy())


def advection_wave(spec: MeshSpec, lev, g, t=0.0, amp=0.5, k=(1, 1, 1)):
    """rho = 1 + amp sin(2 pi sum_d k_d (x_d - v_d t)): smooth and periodic, the
    exact solution of Eq. 13 at time t."""
    X = cell_centres(spec, lev, g)
    s = sum(k[d] * (X[d] - spec.velocity[d] * t) / spec.length[d] for d in range(spec.ndim))
    rho = 1.0 + amp * np.sin(2.0 * np.pi * s)
    return mask_interior(spec, rho.reshape(len(rho), 1, -1).copy())
