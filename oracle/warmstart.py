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
    S = sum_F w^2 |r|^2
    linear:  L = S / (U^2 |F|)          log:  L = log(S / sum_F |b|^2)
with the wall rows of x0 held at their closure values.  Then on fluid rows
    dL/dy = -(2 / (U |F|)) [A^T (w^2 r)]_F      (linear)
    dL/dy = -(2 U / S) [A^T (w^2 r)]_F          (log)
and the targets t = y - (|F| / 2) dL/dy make the mean-squared-error gradient
(2 / |F|)(y - t) equal to dL/dy, so one MSE backward pass through the network
gives dL/dparameters.  Here A^T is the true transpose; the library uses A in its
place, valid because the fluid block of A is symmetric for equal masses (pinned in
the tests).

Pinned by tests/test_oracle_warmstart.py: the wall rows of the residual vanish,
the closure equals the Shepard formula written from the kernel, and the targets'
MSE gradient equals central finite differences of L in parameter space.
"""
import numpy as np

FLUID = 0


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


def start(A, b, v, y, ptype, U):
    """x0 = v + U y on fluid rows, the wall closure on wall rows (y = None: v alone)."""
    fl = np.asarray(ptype) == FLUID
    x = np.array(b, np.float64, copy=True)
    v = np.asarray(v, np.float64)[:, :3]
    x[fl] = v[fl] + (0.0 if y is None else U * np.asarray(y, np.float64)[fl, :3])
    return closure(A, b, x, ptype)


def loss(A, b, x0, ptype, U, jacobi=True, log=True):
    """The residual loss L of x0 (see the module docstring)."""
    fl = np.asarray(ptype) == FLUID
    r = np.asarray(b, np.float64) - A @ x0
    w = 1.0 / A.diagonal() if jacobi else np.ones(A.shape[0])
    S = float(((w[fl, None] * r[fl]) ** 2).sum())
    if log:
        return float(np.log(S / float((np.asarray(b, np.float64)[fl] ** 2).sum())))
    return S / (U * U * int(fl.sum()))


def residual_targets(A, b, v, y, ptype, U, jacobi=True, log=True):
    """Targets t [n, 3] (zero on wall rows), the start x0 and the loss L for network output y."""
    fl = np.asarray(ptype) == FLUID
    nF = int(fl.sum())
    x0 = start(A, b, v, y, ptype, U)
    r = np.asarray(b, np.float64) - A @ x0
    w = 1.0 / A.diagonal() if jacobi else np.ones(A.shape[0])
    z = np.where(fl[:, None], (w * w)[:, None] * r, 0.0)
    S = float(((w[fl, None] * r[fl]) ** 2).sum())
    g = A.T @ z                                  # [A^T (w^2 r)], wall rows of z are zero
    if log:
        dLdy = -(2.0 * U / S) * g
        L = float(np.log(S / float((np.asarray(b, np.float64)[fl] ** 2).sum())))
    else:
        dLdy = -(2.0 / (U * nF)) * g
        L = S / (U * U * nF)
    t = np.zeros((A.shape[0], 3))
    t[fl] = np.asarray(y, np.float64)[fl, :3] - 0.5 * nF * dLdy[fl]
    return t, x0, L
