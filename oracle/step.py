"""One semi-implicit predictor/corrector time step (paper Sec. 3.3), in float64.

TEST INFRASTRUCTURE ONLY (see the package docstring).  It restates, around the
oracle's neighbour sets, A(dt) and linear solve, the parts of the SPH step that
produce the viscous system's right-hand side and move the particles:

* Cole's equation of state (Eq. cole-pressure)
      P(rho) = c0^2 rho0 / zeta ((rho / rho0)^zeta - 1)
  and its inverse for the dummy walls' density.
* The dummy-wall pressure of Eq. dummyP (walls moving at constant velocity,
  a_w = 0):  P_w = (sum_F P_a W_wa + g . sum_F rho_a r_wa W_wa) / sum_F W_wa,
  r_wa = r_w - r_a; an empty fluid sum gives P_w = 0.  rho_w = EOS^-1(P_w).
* The inviscid acceleration and the continuity equation (Eqs. part_NS without
  its viscous term, part_continuity), with grad_b W_ab = |F_ab| (r_a - r_b):
      abar_b   = g - sum_a m_a (P_a / rho_a^2 + P_b / rho_b^2) |F_ab| (r_a - r_b)
      drho_b/dt = sum_a m_a (u_b - u_a) . (r_a - r_b) |F_ab|
  Reading X19: the printed signs (with the printed F <= 0 of Sec. 5.2) would
  make the pressure force attractive and compression lower the density; the
  forms above are the ones under which pressure repels and compression raises
  the density (pinned by the Fourier closed forms in tests/test_oracle_step.py).
  Wall neighbours enter with their prescribed velocity; dummy walls with their
  closure pressure and density.  The acceleration is evaluated on fluid rows;
  the density rate on fluid rows and dynamic wall rows (whose density evolves
  by continuity, Sec. 2.4); dummy walls take theirs from the pressure closure.
* The step (Sec. 3.3): abar^n, drho^n; solve A^n(dt/2) V = B(dt/2) with
  B_fluid = u^n + dt/2 abar^n (walls: 2 u_w dummy, u_w dynamic) for u^{n+1/2};
  r^{n+1/2} = r^n + dt/2 u^n, rho^{n+1/2} = rho^n + dt/2 drho^n, mu^{n+1/2}
  from the Papanastasiou pass at the half state; then abar, drho there; solve
  A^{n+1/2}(dt) V = u^n + dt abar^{n+1/2} for u^{n+1};
  r^{n+1} = r^n + dt/2 (u^n + u^{n+1}), rho^{n+1} = rho^n + dt drho^{n+1/2}.
  Walls move with their prescribed velocity.

Storage follows the state the library keeps: positions, velocities, densities
and viscosities are float32, each update evaluated in float64 (one product,
one sum, no fused operation) and rounded once; positions on periodic axes are
folded back into [lo, hi) in float64 before the rounding.
"""
import numpy as np

from . import kernel, neighbors, operator, rheology, solvers

FLUID = 0


def eos(rho, rho0, c0, zeta):
    rho = np.asarray(rho, np.float64)
    return c0 * c0 * rho0 / zeta * ((rho / rho0) ** zeta - 1.0)


def eos_inverse(P, rho0, c0, zeta):
    P = np.asarray(P, np.float64)
    return rho0 * (P * zeta / (c0 * c0 * rho0) + 1.0) ** (1.0 / zeta)


def _pairs(scene, off, idx):
    b, a = operator.csr_pairs(off, idx)
    P = np.asarray(scene.pos, np.float32)[:, :3].astype(np.float64)
    d = P[a] - P[b]                                   # r_a - r_b
    for ax in range(3):
        if scene.periodic[ax]:
            L = scene.hi[ax] - scene.lo[ax]
            d[:, ax] -= L * np.rint(d[:, ax] / L)
    r = np.sqrt((d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1]) + d[:, 2] * d[:, 2])
    h = float(np.float32(scene.h))
    kid = getattr(scene, "kernel", 0)
    return b, a, d, np.abs(kernel.F(r, h, kid)), kernel.W(r, h, kid)


def wall_closure(scene, off, idx, rho_f, P_f, g, prm):
    """Pressure and density of every particle: fluid (and dynamic walls) from the EOS
    of their density, dummy walls from Eq. dummyP and the inverse EOS."""
    rho = np.asarray(rho_f, np.float64).copy()
    P = np.asarray(P_f, np.float64).copy()
    if scene.boundary != operator.BC_DUMMY:
        return rho, P
    ptype = np.asarray(scene.ptype)
    b, a, d, absF, W = _pairs(scene, off, idx)
    sel = (ptype[b] != FLUID) & (ptype[a] == FLUID)
    n = scene.n
    S = np.zeros(n)
    num = np.zeros(n)
    np.add.at(S, b[sel], W[sel])
    gr = -(d[sel] @ np.asarray(g, np.float64))        # g . (r_w - r_a)
    np.add.at(num, b[sel], P[a[sel]] * W[sel] + gr * rho[a[sel]] * W[sel])
    wall = ptype != FLUID
    Pw = np.where(S > 0, num / np.where(S > 0, S, 1.0), 0.0)
    P[wall] = Pw[wall]
    rho[wall] = eos_inverse(Pw[wall], prm["rho0"], prm["c0"], prm["zeta"])
    return rho, P


def forces(scene, off, idx, rho, P, vel, g):
    """abar (fluid rows) and drho/dt (fluid and dynamic wall rows)."""
    ptype = np.asarray(scene.ptype)
    m = np.asarray(scene.pos, np.float32)[:, 3].astype(np.float64)
    u = np.asarray(vel, np.float32)[:, :3].astype(np.float64)
    b, a, d, absF, _ = _pairs(scene, off, idx)
    n = scene.n
    coef = m[a] * (P[a] / (rho[a] * rho[a]) + P[b] / (rho[b] * rho[b])) * absF
    acc = np.zeros((n, 3))
    np.add.at(acc, b, -coef[:, None] * d)
    acc += np.asarray(g, np.float64)
    acc[ptype != FLUID] = 0.0
    drho = np.zeros(n)
    np.add.at(drho, b, m[a] * np.einsum("ij,ij->i", u[b] - u[a], d) * absF)
    if scene.boundary == operator.BC_DUMMY:
        drho[ptype != FLUID] = 0.0
    return acc, drho


def _advance(scene, base_pos, vel_sum, scale):
    """float32(base + scale * vel_sum) per coordinate, folded on periodic axes."""
    p = np.asarray(base_pos, np.float32)[:, :3].astype(np.float64) + np.asarray(vel_sum, np.float64) * scale
    for ax in range(3):
        if scene.periodic[ax]:
            L = scene.hi[ax] - scene.lo[ax]
            p[:, ax] = np.where(p[:, ax] >= scene.hi[ax], p[:, ax] - L, p[:, ax])
            p[:, ax] = np.where(p[:, ax] < scene.lo[ax], p[:, ax] + L, p[:, ax])
    out = np.asarray(base_pos, np.float32).copy()
    out[:, :3] = p.astype(np.float32)
    return out


def _rhs(scene, u_n, acc, hdt):
    ptype = np.asarray(scene.ptype)
    fl = ptype == FLUID
    uw = np.asarray(scene.wall_vel, np.float32)[:, :3].astype(np.float64)
    b = np.zeros((scene.n, 3))
    b[fl] = u_n[fl] + hdt * acc[fl]
    b[~fl] = (2.0 if scene.boundary == operator.BC_DUMMY else 1.0) * uw[~fl]
    return b


def _evaluate(s, prm, g):
    """Neighbours, viscosity, wall closure, forces of the state s (updated in place:
    the dummy walls' density and, with a rheology, mu)."""
    off, idx = neighbors.build(s.pos, s.lo, s.hi, s.periodic, s.h, kernel_id=getattr(s, "kernel", 0))
    if s.rheology is not None:
        s.mu = rheology.mu_pass(s, off, idx, s.vel)[0].astype(np.float32)
    rho_f = np.asarray(s.rho, np.float32).astype(np.float64)
    rho, P = wall_closure(s, off, idx, rho_f, eos(rho_f, prm["rho0"], prm["c0"], prm["zeta"]), g, prm)
    s.rho = rho.astype(np.float32)
    acc, drho = forces(s, off, idx, s.rho.astype(np.float64), P, s.vel, g)
    return off, idx, acc, drho


def step(scene, prm, rtol=1e-13):
    """One step of Sec. 3.3 on a copy of scene (pos, vel, rho, mu float32; wall rows of
    vel hold the wall velocity).  prm: dt, rho0, c0, zeta, g, and optionally picard
    (>= 0) and picard_tol: with a rheology, the viscosity of the corrector's system
    is recomputed from the new velocities at r^{n+1/2} and the system solved again,
    up to picard times or until ||u_k - u_{k-1}|| / ||u_k|| <= picard_tol over the
    fluid rows (the non-linear form Sec. 8 proposes; picard = 0 keeps the paper's
    lagged viscosity).  Returns the new scene and a dict with the half-step state,
    both solutions (float64) and the fixed-point passes."""
    s = scene.copy()
    dt = float(prm["dt"])
    g = np.asarray(prm["g"], np.float64)
    ptype = np.asarray(s.ptype)
    fl = ptype == FLUID
    r_n = np.asarray(s.pos, np.float32).copy()
    u_n = np.asarray(s.vel, np.float32)[:, :3].astype(np.float64)
    uw = np.asarray(s.wall_vel, np.float32)[:, :3].astype(np.float64)
    # predictor
    off, idx, acc, drho = _evaluate(s, prm, g)
    rho_n = np.asarray(s.rho, np.float32).copy()
    A = operator.assemble(s, off, idx, dt=0.5 * dt)
    B = _rhs(s, u_n, acc, 0.5 * dt)
    x0 = B.copy()
    x0[fl] = u_n[fl]
    u_half = solvers.reference_solution(A, B, x0, rtol=rtol)
    step_v = np.where(fl[:, None], u_n, uw)
    s.pos = _advance(s, r_n, step_v, 0.5 * dt)
    s.rho = (rho_n.astype(np.float64) + drho * (0.5 * dt)).astype(np.float32)
    vel = np.asarray(s.vel, np.float32).copy()
    vel[fl, :3] = u_half[fl].astype(np.float32)
    s.vel = vel
    half = dict(pos=s.pos.copy(), rho=s.rho.copy(), u=u_half.copy(), drho_n=drho.copy(), acc_n=acc.copy())
    # corrector
    off, idx, acc_h, drho_h = _evaluate(s, prm, g)
    half["rho_closed"] = s.rho.copy()
    half["mu"] = np.asarray(s.mu, np.float32).copy()
    A = operator.assemble(s, off, idx, dt=dt)
    B = _rhs(s, u_n, acc_h, dt)
    x0 = B.copy()
    x0[fl] = u_half[fl]
    u_new = solvers.reference_solution(A, B, x0, rtol=rtol)
    passes, change = 0, None
    if s.rheology is not None:
        for _ in range(int(prm.get("picard", 0))):
            vk = np.asarray(s.vel, np.float32).copy()
            vk[fl, :3] = u_new[fl].astype(np.float32)
            mu_k = rheology.mu_pass(s, off, idx, vk)[0]
            s.mu = mu_k.astype(np.float32)
            A = operator.assemble(s, off, idx, dt=dt)
            u_prev = u_new
            u_new = solvers.reference_solution(A, B, u_prev, rtol=rtol)
            passes += 1
            change = np.linalg.norm(u_new[fl] - u_prev[fl]) / np.linalg.norm(u_new[fl])
            if change <= prm.get("picard_tol", 1e-6):
                break
    vsum = np.where(fl[:, None], u_n + u_new, 2.0 * uw)
    s.pos = _advance(s, r_n, vsum, 0.5 * dt)
    # dummy walls have drho = 0: they keep the closure density of step n, which the
    # next step's evaluation recomputes anyway
    s.rho = (rho_n.astype(np.float64) + drho_h * dt).astype(np.float32)
    vel = np.asarray(s.vel, np.float32).copy()
    vel[fl, :3] = u_new[fl].astype(np.float32)
    s.vel = vel
    return s, dict(half=half, u_new=u_new, acc_half=acc_h, drho_half=drho_h, rhs=B, picard_passes=passes,
                   picard_change=change, off=off, idx=idx)
