"""Warm-start x0 and the residual training loss, float64 (test infrastructure only).

The paper starts each solve from the previous velocity (Sec. 4) and names a
better initial guess as future work (Sec. 8).  This module restates what the
library's warm start computes, in plain sparse algebra on the assembled A(dt):

x0 on fluid rows is v + U y, y the network output (y = 0: the previous-step
start), U the RMS of |v| over the fluid.  On a dummy-wall row the system of
Eq. implicit-system-dummy-full reads A_ww x_w + sum over fluid a of A_wa x_a = b_w
(Eq. dummyvel), so x_w = (b_w - sum_a A_wa x_a) / A_ww makes that row of b - A x0
vanish.  A dynamic-wall row is an identity row, so the same formula gives b_w.

Residual loss over the fluid rows F, weight w = 1 / A_bb (Jacobi) or 1,
r = b - A x0:
    R = sum_F w^2 |r|^2
    linear:  L = R / (U^2 |F|)          log:  L = log(R / sum_F |b|^2)
with the wall rows of x0 held at their closure values.  Then on fluid rows
    dL/dy = -(2 / (U |F|)) [A^T (w^2 r)]_F      (linear)
    dL/dy = -(2 U / R) [A^T (w^2 r)]_F          (log)
and the targets t = y - (|F| / 2) dL/dy make the mean-squared-error gradient
(2 / |F|)(y - t) equal to dL/dy, so one MSE backward pass through the network
gives dL/dparameters.  Here A^T is the true transpose; the library uses A in its
place, valid because the fluid block of A is symmetric for equal masses (pinned in
the tests).

High-pass option: x0 = v + U (I - S) y, where (S y)_b = sum_a W_ab V_a y_a /
sum_a W_ab V_a over the fluid neighbours a of b and b itself (V = m / rho):
only the particle-scale part of the correction enters x0.  The targets then
carry P^T = I - S^T in front of A^T (w^2 r).

Pinned by tests/test_oracle_warmstart.py: the wall rows of the residual vanish,
the closure equals the Shepard formula written from the kernel, and the targets'
MSE gradient equals central finite differences of L in parameter space (with and
without the high-pass).
"""
import numpy as np
import scipy.sparse as sp

from . import kernel, neighbors

FLUID = 0


def shepard_matrix(scene, offsets, idx):
    """S (n x n, CSR): on fluid rows b, S_ba = W_ab V_a / sum_c W_cb V_c over a in
    {b} and the fluid neighbours of b; zero rows for walls."""
    n = scene.n
    fl = np.asarray(scene.ptype) == FLUID
    h = float(np.float32(scene.h))
    m = np.asarray(scene.pos, np.float32)[:, 3].astype(np.float64)
    rho = np.asarray(scene.rho, np.float32).astype(np.float64)
    V = m / rho
    rows, cols, vals = [], [], []
    for b in np.flatnonzero(fl):
        nb = np.asarray(idx[offsets[b]:offsets[b + 1]], np.int64)
        nb = nb[fl[nb]]
        r = np.sqrt(neighbors.pair_r2(scene.pos, nb, np.full(nb.shape, b), scene.lo, scene.hi, scene.periodic))
        w = np.concatenate([[kernel.W(0.0, h) * V[b]], kernel.W(r, h) * V[nb]])
        rows.extend([b] * (len(nb) + 1))
        cols.extend([b] + list(nb))
        vals.extend(list(w / w.sum()))
    return sp.csr_matrix((vals, (rows, cols)), shape=(n, n))


def fluid_scale(v, ptype):
    """U = RMS of |v| over the fluid particles."""
    fl = np.asarray(ptype) == FLUID
    v = np.asarray(v, np.float64)[:, :3]
    return float(np.sqrt((v[fl] ** 2).sum() / max(int(fl.sum()), 1)))


def closure(A, b, x0, ptype):
    """x0 with every wall row replaced by (b_w - sum over other columns A_wa x_a) / A_ww."""
    A = A.tocsr()
    x = np.array(x0, np.float64, copy=True)
    wall = np.flatnonzero(np.asarray(ptype) != FLUID)
    diag = A.diagonal()
    for w in wall:
        lo, hi = A.indptr[w], A.indptr[w + 1]
        s = np.zeros(3)
        for k in range(lo, hi):
            a = A.indices[k]
            if a != w:
                s += A.data[k] * x[a]
        x[w] = (np.asarray(b[w], np.float64) - s) / diag[w]
    return x


def start(A, b, v, y, ptype, U, S=None):
    """x0 = v + U y (U (I - S) y with the Shepard matrix S) on fluid rows, the wall
    closure on wall rows (y = None: v alone)."""
    fl = np.asarray(ptype) == FLUID
    x = np.array(b, np.float64, copy=True)
    v = np.asarray(v, np.float64)[:, :3]
    if y is None:
        x[fl] = v[fl]
    else:
        yy = np.asarray(y, np.float64)[:, :3]
        if S is not None:
            yy = yy - S @ yy
        x[fl] = v[fl] + U * yy[fl]
    return closure(A, b, x, ptype)


def loss(A, b, x0, ptype, U, jacobi=True, log=True):
    """The residual loss L of x0 (see the module docstring)."""
    fl = np.asarray(ptype) == FLUID
    r = np.asarray(b, np.float64) - A @ x0
    w = 1.0 / A.diagonal() if jacobi else np.ones(A.shape[0])
    rsum = float(((w[fl, None] * r[fl]) ** 2).sum())
    if log:
        return float(np.log(rsum / float((np.asarray(b, np.float64)[fl] ** 2).sum())))
    return rsum / (U * U * int(fl.sum()))


def residual_targets(A, b, v, y, ptype, U, jacobi=True, log=True, S=None):
    """Targets t [n, 3] (zero on wall rows), the start x0 and the loss L for network
    output y (with the Shepard matrix S: the high-pass start)."""
    fl = np.asarray(ptype) == FLUID
    nF = int(fl.sum())
    x0 = start(A, b, v, y, ptype, U, S)
    r = np.asarray(b, np.float64) - A @ x0
    w = 1.0 / A.diagonal() if jacobi else np.ones(A.shape[0])
    z = np.where(fl[:, None], (w * w)[:, None] * r, 0.0)
    rsum = float(((w[fl, None] * r[fl]) ** 2).sum())
    g = A.T @ z                                  # [A^T (w^2 r)], wall rows of z are zero
    if S is not None:
        g = np.where(fl[:, None], g, 0.0)
        g = g - S.T @ g                          # P^T = I - S^T
    if log:
        dLdy = -(2.0 * U / rsum) * g
        L = float(np.log(rsum / float((np.asarray(b, np.float64)[fl] ** 2).sum())))
    else:
        dLdy = -(2.0 / (U * nF)) * g
        L = rsum / (U * U * nF)
    t = np.zeros((A.shape[0], 3))
    t[fl] = np.asarray(y, np.float64)[fl, :3] - 0.5 * nF * dLdy[fl]
    return t, x0, L
