"""The viscous matrix A(dt) of the semi-implicit step, assembled in float64 (paper Sec. 3.2).

Fluid row beta (Eqs. implicit-system-base, diag, offdiag), with reading X1 (the
gradient factor enters as |F|, which makes the fluid rows strictly diagonally
dominant as the paper states):

    c_ab      = 2 mubar_ab m_a |F_ab| / (rho_a rho_b)          (Eq. kab, |K_ab|)
    A[b, b]   = 1 + dt * sum_a c_ab       (sum over fluid and wall neighbours)
    A[b, a]   = -dt * c_ab

mubar_ab is the harmonic mean 2 mu_a mu_b / (mu_a + mu_b) or the arithmetic mean
(mu_a + mu_b)/2 (Sec. 2.3).  For a wall neighbour a the fluid row's own mu_b is
used, so mubar = mu_b under either mean (reading X6).

Wall row beta:
    dummy  (Eq. implicit-system-dummy-full): A[b, b] = 1, A[b, a] = W_ba / S_b for
           fluid neighbours a, S_b = sum_{a fluid} W_ba; S_b = 0 gives an identity
           row (reading X7)
    dynamic (Eq. implicit-system-dyn-full): identity row

Jacobi preconditioning (App. B) divides each row by its diagonal (left scaling).
"""
import numpy as np
import scipy.sparse as sp

from . import kernel, neighbors

FLUID = 0
WALL = 1
BC_DUMMY = 0
BC_DYNAMIC = 1
MEAN_HARMONIC = 0
MEAN_ARITHMETIC = 1


def csr_pairs(offsets, idx):
    """(row b, neighbour a) index arrays of every CSR entry."""
    n = len(offsets) - 1
    b = np.repeat(np.arange(n, dtype=np.int64), np.diff(offsets))
    return b, np.asarray(idx, dtype=np.int64)


def mean_mu(mu_a, mu_b, mean):
    if mean == MEAN_ARITHMETIC:
        return 0.5 * (mu_a + mu_b)
    return 2.0 * mu_a * mu_b / (mu_a + mu_b)


def pair_terms(scene, b, a, mu=None):
    """For pairs (row b, neighbour a): the fluid-row coefficient c_ab and the kernel W_ab.

    c_ab is defined for every pair; only fluid rows use it.  W_ab is used by
    dummy wall rows.
    """
    r = np.sqrt(neighbors.pair_r2(scene.pos, a, b, scene.lo, scene.hi, scene.periodic))
    mu = np.asarray(scene.mu if mu is None else mu, dtype=np.float32).astype(np.float64)
    rho = np.asarray(scene.rho, dtype=np.float32).astype(np.float64)
    m = np.asarray(scene.pos, dtype=np.float32)[:, 3].astype(np.float64)
    ptype = np.asarray(scene.ptype)
    h = float(np.float32(scene.h))
    kid = getattr(scene, "kernel", 0)
    absF = np.abs(kernel.F(r, h, kid))
    mub = np.where(ptype[a] == FLUID, mean_mu(mu[a], mu[b], scene.mean), mu[b])
    c = 2.0 * mub * m[a] * absF / (rho[a] * rho[b])
    return c, kernel.W(r, h, kid)


def assemble(scene, offsets, idx, dt=None, mu=None, boundary=None):
    """A(dt) as a scipy CSR matrix in float64 (caller order)."""
    n = scene.n
    dt = float(scene.dt if dt is None else dt)
    boundary = scene.boundary if boundary is None else boundary
    ptype = np.asarray(scene.ptype)
    b, a = csr_pairs(offsets, idx)
    c, Wab = pair_terms(scene, b, a, mu)
    fluid_row = ptype[b] == FLUID
    diag = np.ones(n)
    np.add.at(diag, b[fluid_row], dt * c[fluid_row])
    rows, cols, vals = [b[fluid_row]], [a[fluid_row]], [-dt * c[fluid_row]]
    if boundary == BC_DUMMY:
        sel = (~fluid_row) & (ptype[a] == FLUID)
        S = np.zeros(n)
        np.add.at(S, b[sel], Wab[sel])
        bs, as_, ws = b[sel], a[sel], Wab[sel]
        ok = S[bs] > 0.0
        rows.append(bs[ok])
        cols.append(as_[ok])
        vals.append(ws[ok] / S[bs[ok]])
    rows.append(np.arange(n))
    cols.append(np.arange(n))
    vals.append(diag)
    A = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n))
    A.sum_duplicates()
    A.sort_indices()
    return A


def shepard_sums(scene, offsets, idx):
    """S_b = sum over fluid neighbours of W_ba (the denominator of Eq. dummyvel)."""
    b, a = csr_pairs(offsets, idx)
    _, Wab = pair_terms(scene, b, a)
    S = np.zeros(scene.n)
    sel = np.asarray(scene.ptype)[a] == FLUID
    np.add.at(S, b[sel], Wab[sel])
    return S


def jacobi_diag(A):
    return A.diagonal().copy()


def row_norms2(A):
    """Squared Euclidean norms of the rows of D^-1 A, D = diag(A): the Jacobi-scaled
    matrix of App. B, from which a diagonal preconditioner scale is built."""
    A = sp.csr_matrix(A, dtype=np.float64)
    B = sp.diags(1.0 / A.diagonal()) @ A
    return np.asarray(B.multiply(B).sum(axis=1)).ravel()


def wall_row_scale(scene, A, power, factor=1.0):
    """The closed-form row scale: factor row_norms2^-power on the wall rows that carry
    Shepard weights (a fluid neighbour), 1 on fluid rows and on identity rows (lone dummy
    walls and every wall row of a dynamic boundary)."""
    A = sp.csr_matrix(A)
    s = np.ones(scene.n)
    w = (np.asarray(scene.ptype) != FLUID) & (np.diff(A.indptr) > 1)
    s[w] = float(factor) * row_norms2(A)[w] ** (-float(power))
    return s


def apply(A, v):
    """y = A v for an [N, 3] (or [N]) array, in float64."""
    return A @ np.asarray(v, dtype=np.float64)


def true_residual(A, x, b):
    """Joint and per-component relative residual ||b - A x||_2 / ||b||_2 in float64."""
    x = np.asarray(x, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    r = b - A @ x
    nb = np.linalg.norm(b)
    joint = np.linalg.norm(r) / nb if nb > 0 else np.linalg.norm(r)
    per = []
    for c in range(b.shape[1]):
        nbc = np.linalg.norm(b[:, c])
        per.append(np.linalg.norm(r[:, c]) / nbc if nbc > 0 else np.linalg.norm(r[:, c]))
    return joint, np.array(per)


def rows_apply(scene, rows, nbr_rows, x, mu=None):
    """(A x) at selected rows only, each row's neighbour set given (sampled checks at full size).

    Restates the row definitions above one row at a time, so a result at full
    size can be checked without assembling the whole matrix.
    """
    x = np.asarray(x, dtype=np.float64)
    out = np.zeros((len(rows), x.shape[1]))
    for k, (beta, nb) in enumerate(zip(rows, nbr_rows)):
        nb = np.asarray(nb, dtype=np.int64)
        bb = np.full(nb.shape, int(beta), np.int64)
        c, Wab = pair_terms(scene, bb, nb, mu)
        xb = x[beta]
        if scene.ptype[beta] == FLUID:
            out[k] = xb + scene.dt * (c[:, None] * (xb[None, :] - x[nb])).sum(axis=0)
        elif scene.boundary == BC_DUMMY:
            fl = scene.ptype[nb] == FLUID
            S = Wab[fl].sum()
            out[k] = xb + ((Wab[fl][:, None] * x[nb[fl]]).sum(axis=0) / S if S > 0 else 0.0)
        else:
            out[k] = xb
    return out
