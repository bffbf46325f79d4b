"""Features of the learned warm start, float64 (test infrastructure only).

Restates, one feature at a time, the sixteen per-particle inputs of the warm-start
network (the paper names a better initial guess as future work, Sec. 8; the
feature set is this project's choice, listed in the library header):
  0-2  v / U                         U = RMS |v| over the fluid particles
  3-5  e1 / U, e1 = D^-1 (v - A v)   on fluid rows (A = A(dt), D its diagonal)
  6-8  e2 / U, e2 = D^-1 (e1 - A e1) on fluid rows
  9    log10(mu) / 5
  10   log10(D) / 4; on a wall row (D = 1) log10 of the mean D of its fluid neighbours / 4
       (0 without one)
  11   min over wall neighbours of r / (2h), 1 without one
  12   W(0) V_b + sum over fluid neighbours of W_ba V_a (W of the scene's kernel)
  13   neighbour count / 80
  14   |v_b| / (|v_b| + sqrt(mean over neighbours of |v_a|^2))
  15   1 for wall particles
"""
import numpy as np

from . import kernel, neighbors, operator

FLUID = 0


def features(scene, offsets, idx, A, vel=None):
    n = scene.n
    v = np.asarray(scene.vel if vel is None else vel, np.float32)[:, :3].astype(np.float64)
    fl = np.asarray(scene.ptype) == FLUID
    D = A.diagonal()
    U = np.sqrt((v[fl] ** 2).sum() / max(fl.sum(), 1))
    iU = 1.0 / U if U > 0 else 0.0
    e1 = np.where(fl[:, None], (v - A @ v) / D[:, None], 0.0)
    e2 = np.where(fl[:, None], (e1 - A @ e1) / D[:, None], 0.0)
    F = np.zeros((n, 16))
    F[:, 0:3] = v * iU
    F[:, 3:6] = e1 * iU
    F[:, 6:9] = e2 * iU
    F[:, 9] = np.log10(np.asarray(scene.mu, np.float32).astype(np.float64)) / 5.0
    F[:, 10] = np.log10(D) / 4.0
    h = float(np.float32(scene.h))
    kid = getattr(scene, "kernel", kernel.WENDLAND)
    m = np.asarray(scene.pos, np.float32)[:, 3].astype(np.float64)
    rho = np.asarray(scene.rho, np.float32).astype(np.float64)
    V = m / rho
    for b in range(n):
        nb = idx[offsets[b]:offsets[b + 1]].astype(np.int64)
        r = np.sqrt(neighbors.pair_r2(scene.pos, nb, np.full(nb.shape, b), scene.lo, scene.hi, scene.periodic))
        wall = ~fl[nb]
        F[b, 11] = min(1.0, (r[wall] / (2 * h)).min()) if wall.any() else 1.0
        F[b, 12] = kernel.W(0.0, h, kid) * V[b] + (kernel.W(r[~wall], h, kid) * V[nb[~wall]]).sum()
        F[b, 13] = len(nb) / 80.0
        if not fl[b]:
            F[b, 10] = np.log10(D[nb[~wall]].mean()) / 4.0 if (~wall).any() else 0.0
        vn = np.linalg.norm(v[b])
        rms = np.sqrt((v[nb] ** 2).sum(axis=1).mean()) if len(nb) else 0.0
        F[b, 14] = vn / (vn + rms) if vn + rms > 0 else 0.0
    F[:, 15] = (~fl).astype(np.float64)
    return F, U
