"""Shear-rate-dependent viscosity in float64 (paper Sec. 2.1 Eq. papa; Sec. 2.4 "Non-Newtonian viscosity").

For each fluid particle beta, from the velocities of the previous step (the
viscosity is lagged so the system stays linear, Sec. 3.3):

    grad u_beta = sum_a V_a |F_ab| r_ab (x) u_ab,   V_a = m_a / rho_a,
                  r_ab = r_a - r_b, u_ab = u_a - u_b
    gdot        = (grad u + grad u^T) / 2
    D           = sqrt(2 gdot:gdot)                                   (reading X4)
    mu          = tau0 Y(D) + mu0,   Y(D) = (1 - exp(-m D)) / D,  Y(0) = m  (Eq. papa)

|F| follows reading X1 (with the printed signed F the sum is -grad u; D does not
change).  A wall neighbour contributes its prescribed wall velocity u_w (reading
X13).  Y is evaluated as -expm1(-m D)/D in float64.

``series_T`` is the paper's truncated MacLaurin series of (1 - e^{-x})/x in Horner
form (8 terms), used by single-precision code below the switch x = m D < 0.5
(reading X3).
"""
import numpy as np

from . import kernel, neighbors

FLUID = 0


def velocity_gradient(scene, offsets, idx, vel=None):
    """[N, 3, 3] array G with G[b, i, j] = sum_a V_a |F_ab| (r_ab)_i (u_ab)_j; wall rows zero."""
    n = scene.n
    vel = np.asarray(scene.vel if vel is None else vel, dtype=np.float32)[:, :3].astype(np.float64)
    ptype = np.asarray(scene.ptype)
    uw = np.asarray(scene.wall_vel, np.float32)[:, :3].astype(np.float64)
    u = np.where((ptype == FLUID)[:, None], vel, uw)
    b = np.repeat(np.arange(n, dtype=np.int64), np.diff(offsets))
    a = np.asarray(idx, np.int64)
    P = np.asarray(scene.pos, np.float32)[:, :3].astype(np.float64)
    d = P[a] - P[b]
    for ax in range(3):
        if scene.periodic[ax]:
            L = scene.hi[ax] - scene.lo[ax]
            d[:, ax] = d[:, ax] - L * np.rint(d[:, ax] / L)
    r = np.sqrt((d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1]) + d[:, 2] * d[:, 2])
    h = float(np.float32(scene.h))
    absF = np.abs(kernel.F(r, h, getattr(scene, "kernel", 0)))
    V = (np.asarray(scene.pos, np.float32)[:, 3].astype(np.float64)
         / np.asarray(scene.rho, np.float32).astype(np.float64))
    wgt = V[a] * absF
    du = u[a] - u[b]
    G = np.zeros((n, 3, 3))
    contrib = wgt[:, None, None] * d[:, :, None] * du[:, None, :]
    np.add.at(G, b, contrib)
    G[ptype != FLUID] = 0.0
    return G


def shear_rate_invariant(G):
    """D = sqrt(2 gdot:gdot) with gdot = sym(G)."""
    S = 0.5 * (G + np.transpose(G, (0, 2, 1)))
    return np.sqrt(2.0 * np.einsum("nij,nij->n", S, S))


def Y(D, m):
    """(1 - exp(-m D)) / D with the limit m at D = 0."""
    D = np.asarray(D, np.float64)
    safe = np.where(D > 0.0, D, 1.0)
    return np.where(D > 0.0, -np.expm1(-m * safe) / safe, m)


def papanastasiou(D, tau0, mu0, m):
    return tau0 * Y(D, m) + mu0


def series_T(x):
    """T(x) = 1 - x/2 (1 - x/3 (... (1 - x/7 (1 - x/8)) ...)): 8 terms of (1 - e^-x)/x."""
    x = np.asarray(x, np.float64)
    t = np.ones_like(x)
    for k in range(8, 1, -1):
        t = 1.0 - (x / k) * t
    return t


def mu_pass(scene, offsets, idx, vel=None):
    """Per-particle viscosity from the previous velocities (fluid rows; walls keep scene.mu)."""
    tau0, mu0, m = scene.rheology
    G = velocity_gradient(scene, offsets, idx, vel)
    D = shear_rate_invariant(G)
    mu = papanastasiou(D, tau0, mu0, m)
    out = np.asarray(scene.mu, np.float64).copy()
    fl = np.asarray(scene.ptype) == FLUID
    out[fl] = mu[fl]
    return out, D
