"""Seeded synthetic particle scenes for the semi-implicit viscous solve.

This module only lays particles out and draws random numbers.  It holds none of
the method's arithmetic (no kernel, no coefficient, no operator): both the FP64
oracle and the CUDA library receive the arrays built here, so the two share
inputs and nothing else.

Every scene carries exactly what the linear system A(dt) V = B(dt) of the paper
needs (Sec. 3.2, "shared formulation"):

* ``pos``      float32 [N, 4]  x, y, z and the particle mass m (kg) in w
* ``rho``      float32 [N]     density (kg/m^3)
* ``mu``       float32 [N]     dynamic viscosity (Pa s); the paper advises storing
                               mu itself rather than nu*rho (App. A, FMA pitfall)
* ``ptype``    uint8  [N]      0 = fluid, 1 = wall (boundary) particle
* ``wall_vel`` float32 [N, 4]  prescribed wall velocity u_w (xyz; fluid rows ignored)
* ``vel``      float32 [N, 4]  velocity at step n (fluid) / u_w (walls)
* ``b``        float64 [N, 3]  right-hand side B: u^n + dt g for fluid rows,
                               2 u_w for dummy walls, u_w for dynamic walls
* ``x0``       float64 [N, 3]  initial guess (the previous velocity, Sec. 4 /
                               App. B; walls start at their right-hand side)
* ``lo, hi``   float64 [3]     the box; on periodic axes hi - lo is the period
* ``periodic`` int32 [3]
* ``h``        float32         smoothing length
* ``kernel``   int             0 = Wendland (support radius 2h), 1 = truncated
                               Gaussian (support radius 3h), paper Sec. 5.2
* ``dt``       float64         time step of the viscous system

Random draws use numpy's PCG64 seeded with ``SeedSequence([config_id, seed])``.
Lattice positions are (i + 1/2) dx; fluid jitter, where a workload asks for it,
is uniform in +-jitter*dx per coordinate.  Walls are never jittered.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np

FLUID = 0
WALL = 1

BC_DUMMY = 0
BC_DYNAMIC = 1

MEAN_HARMONIC = 0
MEAN_ARITHMETIC = 1

KERNEL_WENDLAND = 0
KERNEL_GAUSSIAN = 1

# config ids used to seed the generators (one stream per workload family)
CFG_COUETTE = 1
CFG_LAVA = 2
CFG_SLOPE = 3
CFG_ENSEMBLE = 4
CFG_LEARNED = 5
CFG_LATTICE = 10
CFG_RANDOM = 11


@dataclasses.dataclass
class Scene:
    name: str
    pos: np.ndarray
    rho: np.ndarray
    mu: np.ndarray
    ptype: np.ndarray
    wall_vel: np.ndarray
    vel: np.ndarray
    b: np.ndarray
    x0: np.ndarray
    lo: np.ndarray
    hi: np.ndarray
    periodic: np.ndarray
    h: float
    dt: float
    boundary: int = BC_DUMMY
    mean: int = MEAN_HARMONIC
    dx: float = 0.0
    # Papanastasiou parameters (tau0, mu0, m) when mu must come from the mu pass
    rheology: Optional[tuple] = None
    meta: dict = dataclasses.field(default_factory=dict)
    kernel: int = KERNEL_WENDLAND

    @property
    def n(self) -> int:
        return int(self.pos.shape[0])

    @property
    def n_fluid(self) -> int:
        return int(np.count_nonzero(self.ptype == FLUID))

    def copy(self) -> "Scene":
        return dataclasses.replace(
            self, **{f.name: (getattr(self, f.name).copy()
                              if isinstance(getattr(self, f.name), np.ndarray) else getattr(self, f.name))
                     for f in dataclasses.fields(self)})

    def with_rhs(self, b: np.ndarray, x0: Optional[np.ndarray] = None) -> "Scene":
        s = self.copy()
        s.b = np.ascontiguousarray(b, dtype=np.float64)
        if x0 is not None:
            s.x0 = np.ascontiguousarray(x0, dtype=np.float64)
        return s


def rng_for(config_id: int, seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence([int(config_id), int(seed)])))


def _lattice(nx, ny, nz, dx, origin=(0.0, 0.0, 0.0)):
    i, j, k = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    p = np.stack([(i.ravel() + 0.5) * dx, (j.ravel() + 0.5) * dx, (k.ravel() + 0.5) * dx], axis=1)
    return p + np.asarray(origin, dtype=np.float64)


def _wrap_periodic(p, lo, hi, periodic):
    p = p.copy()
    for ax in range(3):
        if periodic[ax]:
            L = hi[ax] - lo[ax]
            p[:, ax] = lo[ax] + np.mod(p[:, ax] - lo[ax], L)
    return p


def _assemble(name, fluid_p, wall_p, wall_u, dx, rho0, mu_fluid, dt, lo, hi, periodic,
              v_fluid, g=(0.0, 0.0, 0.0), boundary=BC_DUMMY, mean=MEAN_HARMONIC,
              h_factor=1.3, rheology=None, meta=None, kernel=KERNEL_WENDLAND):
    """Stack fluid and wall particles into a Scene (fluid first, walls after)."""
    nf, nw = fluid_p.shape[0], wall_p.shape[0]
    n = nf + nw
    lo = np.asarray(lo, np.float64)
    hi = np.asarray(hi, np.float64)
    periodic = np.asarray(periodic, np.int32)
    pos64 = np.concatenate([fluid_p, wall_p], axis=0)
    pos64 = _wrap_periodic(pos64, lo, hi, periodic)
    pos = np.zeros((n, 4), np.float32)
    pos[:, :3] = pos64.astype(np.float32)
    # a float32 cast can land exactly on hi on a periodic axis: fold it back
    for ax in range(3):
        if periodic[ax]:
            at_hi = pos[:, ax] >= np.float32(hi[ax])
            pos[at_hi, ax] = np.float32(lo[ax])
    mass = np.float32(rho0 * dx ** 3)
    pos[:, 3] = mass
    rho = np.full(n, rho0, np.float32)
    mu = np.empty(n, np.float32)
    mu[:nf] = np.asarray(mu_fluid, np.float32) if np.ndim(mu_fluid) else np.float32(mu_fluid)
    # wall mu never enters the operator (the fluid row's own mu is used for
    # fluid-wall pairs); keep a finite placeholder
    mu[nf:] = mu[:nf].mean() if nf else np.float32(1.0)
    ptype = np.zeros(n, np.uint8)
    ptype[nf:] = WALL
    wall_vel = np.zeros((n, 4), np.float32)
    wall_vel[nf:, :3] = np.asarray(wall_u, np.float32)
    vel = np.zeros((n, 4), np.float32)
    vel[:nf, :3] = v_fluid.astype(np.float32)
    vel[nf:, :3] = wall_vel[nf:, :3]
    g = np.asarray(g, np.float64)
    b = np.zeros((n, 3), np.float64)
    b[:nf] = vel[:nf, :3].astype(np.float64) + dt * g
    if boundary == BC_DUMMY:
        b[nf:] = 2.0 * wall_vel[nf:, :3].astype(np.float64)
    else:
        b[nf:] = wall_vel[nf:, :3].astype(np.float64)
    x0 = np.zeros((n, 3), np.float64)
    x0[:nf] = vel[:nf, :3].astype(np.float64)
    x0[nf:] = b[nf:]
    return Scene(name=name, pos=pos, rho=rho, mu=mu, ptype=ptype, wall_vel=wall_vel, vel=vel,
                 b=b, x0=x0, lo=lo, hi=hi, periodic=periodic,
                 h=float(np.float32(h_factor * dx)), dt=float(dt), boundary=boundary, mean=mean,
                 dx=float(dx), rheology=rheology, meta=dict(meta or {}), kernel=int(kernel))


def couette(seed: int = 0, nx: int = 20, ny: int = 10, nz: int = 10, dx: float = 0.01,
            rho0: float = 1000.0, nu: float = 1.0, dt: float = 1e-4, U: float = 1.0,
            noise: float = 0.01, layers: int = 3, boundary: int = BC_DUMMY,
            kernel: int = KERNEL_WENDLAND, h_factor: float = 1.3) -> Scene:
    """Plane Couette channel: fluid between two walls normal to y, periodic in x, z.

    Fluid at y = (j + 1/2) dx, j < ny (channel height H = ny dx); wall layers at
    -(k + 1/2) dx and H + (k + 1/2) dx.  With dummy walls the analytical wall sits
    half a spacing from the first wall layer (Sec. 5.1).  Bottom wall at rest,
    top wall moving at (U, 0, 0).  Fluid velocity: the linear profile U y / H plus
    uniform noise of +-noise from the seed.
    """
    H = ny * dx
    fluid = _lattice(nx, ny, nz, dx)
    # both boundary models use the same layout here; the model only changes the
    # wall rows of the operator
    bot = [_lattice(nx, 1, nz, dx, origin=(0.0, -(k + 1) * dx, 0.0)) for k in range(layers)]
    top = [_lattice(nx, 1, nz, dx, origin=(0.0, H + k * dx, 0.0)) for k in range(layers)]
    bot = np.concatenate(bot)
    top = np.concatenate(top)
    walls = np.concatenate([bot, top])
    wall_u = np.zeros((walls.shape[0], 3))
    wall_u[bot.shape[0]:, 0] = U
    rng = rng_for(CFG_COUETTE, seed)
    v = np.zeros((fluid.shape[0], 3))
    v[:, 0] = U * fluid[:, 1] / H
    v += rng.uniform(-noise, noise, size=v.shape)
    lo = (0.0, -layers * dx, 0.0)
    hi = (nx * dx, H + layers * dx, nz * dx)
    return _assemble("couette", fluid, walls, wall_u, dx, rho0, rho0 * nu, dt, lo, hi, (1, 0, 1),
                     v, boundary=boundary, meta=dict(seed=seed, U=U, H=H, nu=nu), kernel=kernel,
                     h_factor=h_factor)


def poiseuille(boundary: int = BC_DUMMY, kernel: int = KERNEL_WENDLAND, inv_dp: int = 16,
               L: float = 1.0, mu: float = 0.1, dt: float = 1e-2, h_factor: float = 1.3) -> Scene:
    """Plane Poiseuille channel of width L at rest, laid out as Sec. 5.2 does for each
    boundary model (rho0 = 1 kg/m^3, h = h_factor dp).

    Dummy walls: the analytical walls lie half a spacing outside the fluid, so
    1/dp fluid layers fill the channel.  Dynamic walls: the first wall layer sits on
    the analytical wall, so 1/dp - 1 fluid layers sit between the two first wall
    layers, one of them on the centre line.  Wall layers: as many as the kernel's
    support reaches (ceil(support / dp): 3 for Wendland at h = 1.3 dp, 4 for the
    truncated Gaussian, 5 for Wendland at h = 2.5 dp).  meta: L and "centre" (the y
    of the centre line; the analytical profile is a function of y - centre).  The
    periodic x and z extent is at least three supports, rounded up to a multiple of
    4 spacings (8, 12 and 16).
    """
    dx = L / inv_dp
    gauss = kernel == KERNEL_GAUSSIAN
    support = (3.0 if gauss else 2.0) * h_factor        # in spacings
    ny = inv_dp if boundary == BC_DUMMY else inv_dp - 1
    layers = int(math.ceil(support - 1e-9))
    nxz = 4 * int(math.ceil(3.0 * support / 4.0 - 1e-9))   # at least three neighbour-grid cells per period
    s = couette(0, nx=nxz, ny=ny, nz=nxz, dx=dx, rho0=1.0, nu=mu, dt=dt, U=0.0, noise=0.0,
                layers=layers, boundary=boundary, kernel=kernel, h_factor=h_factor)
    s.name = "poiseuille"
    s.meta.update(L=L, centre=0.5 * ny * dx)
    return s


def lava_box(seed: int = 0, n: int = 100, dx: float = 0.005, rho0: float = 1000.0, nu: float = 10.0,
             dt: float = 5e-4, sigma: float = 0.1, jitter: float = 0.1, layers: int = 3,
             boundary: int = BC_DUMMY, kernel: int = KERNEL_WENDLAND) -> Scene:
    """Lava-like open box: an n^3 jittered fluid lattice on a dummy floor and four side walls.

    Floor: (n + 2 layers)^2 x layers particles below z = 0; side walls normal to x
    span the full width with the corner columns, walls normal to y span the fluid
    width; both are n particles high.  The top is a free surface.  Fluid
    velocities are N(0, sigma^2) per component; walls at rest; no body force.
    """
    L = n * dx
    rng = rng_for(CFG_LAVA, seed)
    fluid = _lattice(n, n, n, dx)
    fluid = fluid + rng.uniform(-jitter * dx, jitter * dx, size=fluid.shape)
    m = n + 2 * layers
    floor = _lattice(m, m, layers, dx, origin=(-layers * dx, -layers * dx, -layers * dx))
    wx0 = _lattice(layers, m, n, dx, origin=(-layers * dx, -layers * dx, 0.0))
    wx1 = _lattice(layers, m, n, dx, origin=(L, -layers * dx, 0.0))
    wy0 = _lattice(n, layers, n, dx, origin=(0.0, -layers * dx, 0.0))
    wy1 = _lattice(n, layers, n, dx, origin=(0.0, L, 0.0))
    walls = np.concatenate([floor, wx0, wx1, wy0, wy1])
    v = rng.normal(0.0, sigma, size=fluid.shape)
    lo = (-layers * dx, -layers * dx, -layers * dx)
    hi = (L + layers * dx, L + layers * dx, L + 4 * dx)
    return _assemble("lava_box", fluid, walls, np.zeros((walls.shape[0], 3)), dx, rho0, rho0 * nu, dt,
                     lo, hi, (0, 0, 0), v, boundary=boundary, meta=dict(seed=seed, n=n, nu=nu), kernel=kernel)


def slope(seed: int = 0, nx: int = 200, ny: int = 100, nz: int = 200, dx: float = 0.005,
          rho0: float = 1000.0, tau0: float = 100.0, mu0: float = 1e3, m_reg: float = 1000.0,
          dt: float = 5e-4, U: float = 0.1, plug: float = 1.0 / 3.0, noise: float = 1e-5,
          jitter: float = 0.1, theta_deg: float = 10.0, layers: int = 3, boundary: int = BC_DUMMY) -> Scene:
    """Slope flow of a Papanastasiou (regularised Bingham) fluid on an inclined floor.

    The incline is a flat floor normal to y, periodic in x and z, with gravity
    rotated by theta (x downslope).  The seeded velocity is a Bingham-like
    profile: a sheared layer u_x = U (1 - (1 - y/y0)^2) below y0 = (1 - plug) H
    and a rigid plug u_x = U above it, times (1 + noise N(0,1)), plus transverse
    components noise U N(0,1).  |du/dy| runs from 2U/y0 at the floor to 0 in the
    plug, so the viscosity spans [mu(2U/y0), m tau0 + mu0] (about 1e3 to 1e5 Pa s
    with the defaults).  ``mu`` is left at the plateau value; the mu pass fills
    it from ``vel``.
    """
    H = ny * dx
    y0 = (1.0 - plug) * H
    rng = rng_for(CFG_SLOPE, seed)
    fluid = _lattice(nx, ny, nz, dx)
    fluid = fluid + rng.uniform(-jitter * dx, jitter * dx, size=fluid.shape)
    floor = _lattice(nx, layers, nz, dx, origin=(0.0, -layers * dx, 0.0))
    yy = np.clip(fluid[:, 1], 0.0, y0)
    v = np.zeros_like(fluid)
    v[:, 0] = U * (1.0 - (1.0 - yy / y0) ** 2) * (1.0 + noise * rng.standard_normal(fluid.shape[0]))
    v[:, 1] = noise * U * rng.standard_normal(fluid.shape[0])
    v[:, 2] = noise * U * rng.standard_normal(fluid.shape[0])
    th = math.radians(theta_deg)
    g = (9.81 * math.sin(th), -9.81 * math.cos(th), 0.0)
    lo = (0.0, -layers * dx, 0.0)
    hi = (nx * dx, H + 4 * dx, nz * dx)
    mu_plateau = m_reg * tau0 + mu0
    return _assemble("slope", fluid, floor, np.zeros((floor.shape[0], 3)), dx, rho0, mu_plateau, dt,
                     lo, hi, (1, 0, 1), v, g=g, boundary=boundary, rheology=(tau0, mu0, m_reg),
                     meta=dict(seed=seed, U=U, H=H, y0=y0))


def slope_subset(seed: int = 0, **kw) -> Scene:
    """The 50 x 20 x 50 subset of the slope workload (about 57.5k particles)."""
    kw.setdefault("nx", 50)
    kw.setdefault("ny", 20)
    kw.setdefault("nz", 50)
    return slope(seed, **kw)


def periodic_lattice(n: int = 8, dx: float = 0.01, rho0: float = 1000.0, nu: float = 1.0,
                     dt: float = 1e-4, jitter: float = 0.0, seed: int = 0, sigma: float = 0.1,
                     aniso=(1, 1, 1), mu_spread: float = 0.0, kernel: int = KERNEL_WENDLAND) -> Scene:
    """Fluid-only cube periodic on all three axes (no walls).

    With jitter = 0 and uniform mu, rho, m the operator is circulant (Fourier pin).
    ``mu_spread`` > 0 draws mu log-uniformly in [mu, mu * (1 + mu_spread)].
    """
    nxyz = [n * a for a in aniso]
    rng = rng_for(CFG_LATTICE, seed)
    fluid = _lattice(*nxyz, dx)
    if jitter:
        fluid = fluid + rng.uniform(-jitter * dx, jitter * dx, size=fluid.shape)
    v = rng.normal(0.0, sigma, size=fluid.shape)
    mu = np.full(fluid.shape[0], rho0 * nu)
    if mu_spread:
        mu = mu * np.exp(rng.uniform(0.0, math.log1p(mu_spread), size=mu.shape))
    lo = (0.0, 0.0, 0.0)
    hi = tuple(k * dx for k in nxyz)
    return _assemble("periodic_lattice", fluid, np.zeros((0, 3)), np.zeros((0, 3)), dx, rho0, mu, dt,
                     lo, hi, (1, 1, 1), v, kernel=kernel)


def random_box(seed: int = 0, nf: int = 200, nw_layers: int = 2, dx: float = 0.01, rho0: float = 1000.0,
               nu: float = 1.0, dt: float = 1e-4, periodic=(1, 0, 1), boundary: int = BC_DUMMY,
               mean: int = MEAN_HARMONIC, mu_spread: float = 0.0, mass_spread: float = 0.0,
               kernel: int = KERNEL_WENDLAND) -> Scene:
    """Small irregular scene: random fluid positions in a slab over a wall floor.

    Used for exhaustive small-N checks (neighbour sets, operator rows, solves):
    positions are uniform random (not a lattice), so pair distances take generic
    values, masses and viscosities may vary per particle.
    """
    rng = rng_for(CFG_RANDOM, seed)
    side = max(3.0, round((nf / 0.9) ** (1.0 / 3.0)))
    Lx = Lz = side * dx
    Ly = side * dx
    fluid = np.stack([rng.uniform(0, Lx, nf), rng.uniform(0, Ly, nf), rng.uniform(0, Lz, nf)], axis=1)
    nxw = int(round(Lx / dx))
    floor = _lattice(nxw, nw_layers, nxw, dx, origin=(0.0, -nw_layers * dx, 0.0))
    walls = floor
    wall_u = np.zeros((walls.shape[0], 3))
    wall_u[:, 2] = 0.3
    v = rng.normal(0.0, 0.1, size=fluid.shape)
    mu = np.full(nf, rho0 * nu)
    if mu_spread:
        mu = mu * np.exp(rng.uniform(0.0, math.log1p(mu_spread), size=nf))
    lo = (0.0, -nw_layers * dx, 0.0)
    hi = (Lx, Ly + 2 * dx, Lz)
    # periodic lengths must be at least three cells of side 2h
    s = _assemble("random_box", fluid, walls, wall_u, dx, rho0, mu, dt, lo, hi, periodic, v,
                  boundary=boundary, mean=mean, kernel=kernel)
    if mass_spread:
        s.pos[:, 3] *= np.exp(rng.uniform(0.0, math.log1p(mass_spread), size=s.n)).astype(np.float32)
    return s


def stirring_force(scene: Scene, G: float = 160.0) -> np.ndarray:
    """A fixed smooth body force per particle, G (sin 2pi y/L, sin 2pi z/L, sin 2pi x/L) on fluid rows.

    Used by warm-started sequences so that the velocity field settles to a
    steady stirred state instead of decaying to zero (with nu = 10 m^2/s and a
    0.5 m box, G = 160 m/s^2 gives velocities of order 0.1 m/s).
    """
    P = scene.pos[:, :3].astype(np.float64)
    L = np.where(scene.hi - scene.lo > 0, scene.hi - scene.lo, 1.0)
    f = np.zeros((scene.n, 3))
    f[:, 0] = G * np.sin(2 * np.pi * (P[:, 1] - scene.lo[1]) / L[1])
    f[:, 1] = G * np.sin(2 * np.pi * (P[:, 2] - scene.lo[2]) / L[2])
    f[:, 2] = G * np.sin(2 * np.pi * (P[:, 0] - scene.lo[0]) / L[0])
    f[scene.ptype != FLUID] = 0.0
    return f


def _couette_count(ny, layers=3):
    nx = nz = 2 * ny
    return nx * ny * nz + 2 * layers * nx * nz


def _box_count(n, layers=3):
    m = n + 2 * layers
    return n ** 3 + m * m * layers + 2 * layers * m * n + 2 * layers * n * n


def ensemble(seed: int = 0, S: int = 64, n_lo: float = 1e4, n_hi: float = 5e5, dx: float = 0.005,
             nu_lo: float = 1.0, nu_hi: float = 1e3, dt_lo: float = 1e-4, dt_hi: float = 5e-4,
             rho0: float = 1000.0):
    """Independent scenes of log-uniform particle counts, nu and dt (channel / box alternating).

    The drawn count is the scene's total (fluid + wall particles): the lattice
    size whose total is closest to it is used, so the ensemble totals about
    S * (n_hi - n_lo) / ln(n_hi / n_lo) particles (8.0M for the defaults).
    """
    rng = rng_for(CFG_ENSEMBLE, seed)
    scenes = []
    for s in range(S):
        target = math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))
        nu = math.exp(rng.uniform(math.log(nu_lo), math.log(nu_hi)))
        dt = math.exp(rng.uniform(math.log(dt_lo), math.log(dt_hi)))
        sub = int(rng.integers(0, 2**31 - 1))
        if s % 2 == 0:
            ny = min(range(6, 200), key=lambda k: abs(_couette_count(k) - target))
            sc = couette(sub, nx=2 * ny, ny=ny, nz=2 * ny, dx=dx, rho0=rho0, nu=nu, dt=dt, U=1.0, noise=0.01)
        else:
            n = min(range(8, 400), key=lambda k: abs(_box_count(k) - target))
            sc = lava_box(sub, n=n, dx=dx, rho0=rho0, nu=nu, dt=dt)
        sc.name = f"ensemble[{s}]:{sc.name}"
        sc.meta.update(nu=nu, dt=dt, target=target)
        scenes.append(sc)
    return scenes
