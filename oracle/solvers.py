"""Linear solvers of paper Sec. 4, in float64 (optionally float32 vectors with float64 dots).

* ``bicgstab_textbook``  the standard BiCGSTAB as the paper states it (Sec. 4.2,
  first listing): gamma_0 = alpha_0 = omega_0 = 1, p_0 = 0, one system at a time.
* ``bicgstab_paper``     the restructured BiCGSTAB (Sec. 4.2, second listing):
  alpha' = gamma_{i+1}/delta_i and beta = alpha'/omega computed at the end of the
  loop, p_i = r + beta p - alpha' A p, the three velocity components solved
  together with the per-component converged / stalled / progressing states of
  the "Stopping criterion" paragraph and the single exit point.  Optional left
  Jacobi scaling (App. B), merged reductions (the two identities
  gamma' = r0^.r* - omega r0^.Ar* and |r|^2 = |r*|^2 - 2 omega r*.Ar* + omega^2 |Ar*|^2),
  and float32 vector storage to mimic a single-precision implementation.
* ``cg_rotated``         the rotated CG (Sec. 4.1, second listing), optionally
  preconditioned with the Jacobi diagonal (z = D^-1 r, App. B).
* ``dense_solve``        numpy's LU (library routine) on the dense matrix.
* ``gauss_elim``         Gaussian elimination with partial pivoting, by hand.

Tolerance (Sec. 4.1, reading X2): tau^2 = max(eps^2 b.b, FLT_MIN), FLT_MIN = 2^-126
not squared, b the (scaled) right-hand side of the component.
"""
import numpy as np
import scipy.sparse as sp

FLT_MIN = 2.0 ** -126

CONVERGED = 0
STALLED = 1
PROGRESSING = 2


def _dot(u, v):
    return float(np.dot(np.asarray(u, np.float64), np.asarray(v, np.float64)))


def _coldots(U, V):
    return np.einsum("ij,ij->j", np.asarray(U, np.float64), np.asarray(V, np.float64))


def tau2(bb, eps):
    return np.maximum(eps * eps * np.asarray(bb, np.float64), FLT_MIN)


def bicgstab_textbook(A, b, x0=None, eps=1e-12, maxit=10000, jacobi=False):
    """Standard BiCGSTAB on each column of b separately.

    Convergence is checked after each of the two x updates (r . r < tau^2);
    returns (x, iterations per column).
    """
    A = sp.csr_matrix(A)
    b = np.asarray(b, np.float64)
    if b.ndim == 1:
        b = b[:, None]
    n, k = b.shape
    x0 = np.zeros_like(b) if x0 is None else np.asarray(x0, np.float64).reshape(n, k)
    if jacobi:
        D = A.diagonal()
        A = sp.diags(1.0 / D) @ A
        b = b / D[:, None]
    X = x0.copy()
    its = np.zeros(k, np.int64)
    for c in range(k):
        x = X[:, c].copy()
        r = b[:, c] - A @ x
        rh = r.copy()
        t2 = float(tau2(_dot(b[:, c], b[:, c]), eps))
        if _dot(r, r) < t2:
            X[:, c] = x
            continue
        gam_prev = alpha = omega = 1.0
        p = np.zeros(n)
        Ap = np.zeros(n)
        for i in range(1, maxit + 1):
            gam = _dot(rh, r)
            beta = (gam / gam_prev) * (alpha / omega)
            p = r + beta * (p - omega * Ap)
            Ap = A @ p
            delta = _dot(rh, Ap)
            if delta == 0.0 or not np.isfinite(delta):
                break                      # breakdown: the textbook method stalls here
            alpha = gam / delta
            rs = r - alpha * Ap
            xs = x + alpha * p
            its[c] = i
            if _dot(rs, rs) < t2:
                x = xs
                break
            As = A @ rs
            AA = _dot(As, As)
            if AA == 0.0:
                x = xs
                break
            omega = _dot(rs, As) / AA
            r = rs - omega * As
            x = xs + omega * rs
            gam_prev = gam
            if _dot(r, r) < t2:
                break
        X[:, c] = x
    return X, its


class PaperResult:
    def __init__(self, x, iters, state, history, stalled_any=None):
        self.x = x
        self.iters = iters
        self.state = state
        self.history = history
        self.stalled_any = stalled_any


# ---- scalar side of the restructured BiCGSTAB (Sec. 4.2, "Stopping criterion") ----
# One function per point of the iteration where a reduction completes; each works
# component by component in float64.  Reading X8 of "any of the coefficients
# zeroes out": a delta that is zero or not finite, or an alpha that is not
# finite, stalls the component; an omega whose denominator Ar*.Ar* is not a
# positive finite number, or whose quotient is not finite, is zero; alpha' and
# beta are zero after a stall or a zero omega, and both are zero when either is
# not finite; the state is then converged (r.r < tau^2, checked first), stalled
# (a stall this iteration, omega = 0, or r.r not finite) or progressing.
# Components that are not live (frozen) keep every scalar and their state.

def scalar_after_delta(delta, gam, live):
    """alpha = gamma / delta per component; returns (alpha, stall_now)."""
    k = len(gam)
    alpha = np.zeros(k)
    stall = np.zeros(k, bool)
    with np.errstate(all="ignore"):
        for c in range(k):
            if not live[c]:
                continue
            d = np.float64(delta[c])
            if d == 0.0 or not np.isfinite(d):
                stall[c] = True
                continue
            a = np.float64(gam[c]) / d
            if not np.isfinite(a):
                stall[c] = True
                continue
            alpha[c] = a
    return alpha, stall


def scalar_after_omega(sA, AA, live):
    """omega = (r*.Ar*) / (Ar*.Ar*) per component, zero when it cannot be formed."""
    k = len(sA)
    omega = np.zeros(k)
    with np.errstate(all="ignore"):
        for c in range(k):
            if not live[c]:
                continue
            den = np.float64(AA[c])
            if not (den > 0.0 and np.isfinite(den)):
                continue
            om = np.float64(sA[c]) / den
            omega[c] = om if np.isfinite(om) else 0.0
    return omega


def scalar_after_update(state, stall_now, omega, delta, gam, gam_n, rr, t2, live):
    """alpha' = gamma'/delta, beta = alpha'/omega and the new states.

    Returns (alpha_p, beta, gamma, state): gamma and the state change only on
    live components."""
    k = len(gam)
    alpha_p = np.zeros(k)
    beta = np.zeros(k)
    gam_out = np.array(gam, np.float64, copy=True)
    st_out = np.array(state, copy=True)
    with np.errstate(all="ignore"):
        for c in range(k):
            if not live[c]:
                continue
            ok = (not stall_now[c]) and omega[c] != 0.0
            ap = np.float64(gam_n[c]) / np.float64(delta[c]) if ok else 0.0
            be = ap / np.float64(omega[c]) if ok else 0.0
            if not (np.isfinite(ap) and np.isfinite(be)):
                ap = be = 0.0
            alpha_p[c] = ap
            beta[c] = be
            gam_out[c] = gam_n[c]
            r2 = np.float64(rr[c])
            if r2 < t2[c]:
                st_out[c] = CONVERGED
            elif stall_now[c] or omega[c] == 0.0 or not np.isfinite(r2):
                st_out[c] = STALLED
            else:
                st_out[c] = PROGRESSING
    return alpha_p, beta, gam_out, st_out


def bicgstab_paper(A, b, x0=None, eps=2.0 ** -23, maxit=10000, jacobi=True, merged=False,
                   dtype=np.float64, freeze_done=False, record=False):
    """Restructured BiCGSTAB on all columns of b at once (paper Sec. 4.2).

    Vectors are kept in ``dtype``; every dot product and scalar is float64.  With
    ``freeze_done`` a converged or stalled component keeps its x and r (its
    alpha and omega are zero); without it every component runs every iteration
    as the paper describes.  Returns a PaperResult with x (float64), the
    iteration count, the final per-component state, whether each component
    stalled at some iteration and, if ``record``, one dict per iteration with
    x, r.r, the state and the raw dots and scalars of that iteration (delta,
    alpha, r*.Ar*, Ar*.Ar*, omega, gamma', alpha', beta, live).
    """
    A = sp.csr_matrix(A, dtype=np.float64)
    b = np.asarray(b, np.float64)
    if b.ndim == 1:
        b = b[:, None]
    n, k = b.shape
    x0 = np.zeros_like(b) if x0 is None else np.asarray(x0, np.float64).reshape(n, k)
    if jacobi:
        D = A.diagonal()
        A = sp.diags(1.0 / D) @ A
        b = b / D[:, None]

    def mv(v):
        return (A @ np.asarray(v, np.float64)).astype(dtype)

    x = x0.astype(dtype)
    r = (b - A @ x0).astype(dtype)
    rh = r.copy()
    bb = _coldots(b, b)
    t2 = tau2(bb, eps)
    gam = _coldots(rh, r)
    alpha_p = np.zeros(k)
    beta = np.zeros(k)
    rr = _coldots(r, r)
    state = np.where((bb == 0.0) | (rr < t2), CONVERGED, PROGRESSING)
    stalled_any = np.zeros(k, bool)
    p = np.zeros((n, k), dtype)
    Ap = np.zeros((n, k), dtype)
    hist = []
    it = 0
    while np.any(state == PROGRESSING) and it < maxit:
        it += 1
        live = (state == PROGRESSING) if freeze_done else np.ones(k, bool)
        # p_i = r + beta p - alpha' A p; a zero coefficient skips its vector (App. B axpby)
        pn = r.astype(np.float64)
        for c in range(k):
            if beta[c] != 0.0:
                pn[:, c] += beta[c] * p[:, c].astype(np.float64)
            if alpha_p[c] != 0.0:
                pn[:, c] -= alpha_p[c] * Ap[:, c].astype(np.float64)
        p = pn.astype(dtype)
        Ap = mv(p)
        delta = _coldots(rh, Ap)
        alpha, stall_now = scalar_after_delta(delta, gam, live)
        rs = (r.astype(np.float64) - alpha * Ap.astype(np.float64)).astype(dtype)
        xs = x.astype(np.float64) + alpha * p.astype(np.float64)
        As = mv(rs)
        s_AA = _coldots(As, As)
        s_sA = _coldots(rs, As)
        omega = scalar_after_omega(s_sA, s_AA, live)
        if merged:
            s_hs = _coldots(rh, rs)
            s_hA = _coldots(rh, As)
            s_ss = _coldots(rs, rs)
        r = (rs.astype(np.float64) - omega * As.astype(np.float64)).astype(dtype)
        x = (xs + omega * rs.astype(np.float64)).astype(dtype)
        if merged:
            gam_n = s_hs - omega * s_hA
            rr = s_ss - 2.0 * omega * s_sA + omega * omega * s_AA
        else:
            gam_n = _coldots(rh, r)
            rr = _coldots(r, r)
        alpha_p, beta, gam, state = scalar_after_update(state, stall_now, omega, delta, gam, gam_n, rr, t2,
                                                        live)
        stalled_any |= state == STALLED
        if record:
            hist.append(dict(x=x.astype(np.float64).copy(), rr=np.array(rr, np.float64), state=state.copy(),
                             delta=np.array(delta), alpha=alpha.copy(), sA=np.array(s_sA), AA=np.array(s_AA),
                             omega=omega.copy(), gam_n=np.array(gam_n, np.float64), alpha_p=alpha_p.copy(),
                             beta=beta.copy(), live=live.copy()))
    return PaperResult(x.astype(np.float64), it, state, hist, stalled_any)


def cg_rotated(A, b, x0=None, eps=2.0 ** -23, maxit=10000, jacobi=False, record=False):
    """Rotated CG of Sec. 4.1 on each column: p update first, beta and the check last.

    Per iteration i: p_i = z_i + beta_i p_{i-1} (beta_0 = 0, so p_{-1} is never read),
    alpha_i = r_i.z_i / p_i.A p_i, r_{i+1} = r_i - alpha_i A p_i,
    x_{i+1} = x_i + alpha_i p_i, beta_{i+1} = r_{i+1}.z_{i+1} / r_i.z_i, and the
    column is converged when r_{i+1}.r_{i+1} < tau^2 (tau^2 from the column's b).
    Without ``jacobi`` z = r (the printed listing); with it z = D^-1 r, the Jacobi
    preconditioner of App. B applied so that the iteration stays symmetric.
    "Stopping criterion": alpha = 0 in finite precision while r.r >= tau^2 is a
    stall (a zero or non-finite p.Ap, or a non-finite alpha, gives alpha = 0); the
    iteration completes and the column exits.  Returns (x, iterations per column);
    with ``record`` also the final states and, per column, x after each iteration.
    """
    A = sp.csr_matrix(A, dtype=np.float64)
    b = np.asarray(b, np.float64)
    if b.ndim == 1:
        b = b[:, None]
    n, k = b.shape
    w = 1.0 / A.diagonal() if jacobi else np.ones(n)
    X = np.zeros_like(b) if x0 is None else np.asarray(x0, np.float64).reshape(n, k).copy()
    its = np.zeros(k, np.int64)
    states = np.full(k, CONVERGED)
    hist = [[] for _ in range(k)]
    with np.errstate(all="ignore"):
        for c in range(k):
            x = X[:, c]
            r = b[:, c] - A @ x
            t2 = float(tau2(_dot(b[:, c], b[:, c]), eps))
            z = w * r
            gam = _dot(r, z)
            rr = _dot(r, r)
            beta = 0.0
            p = None
            i = 0
            state = CONVERGED if rr < t2 else PROGRESSING
            while state == PROGRESSING and i < maxit:
                p = z.copy() if beta == 0.0 else z + beta * p
                Ap = A @ p
                pAp = _dot(p, Ap)
                alpha = np.float64(gam) / np.float64(pAp) if (pAp != 0.0 and np.isfinite(pAp)) else 0.0
                if not np.isfinite(alpha):
                    alpha = 0.0
                stall = alpha == 0.0
                r = r - alpha * Ap
                x = x + alpha * p
                z = w * r
                gam_n = _dot(r, z)
                rr = _dot(r, r)
                beta = 0.0 if stall else np.float64(gam_n) / np.float64(gam)
                if not np.isfinite(beta):
                    beta = 0.0
                gam = gam_n
                i += 1
                if rr < t2:
                    state = CONVERGED
                elif stall or not np.isfinite(rr):
                    state = STALLED
                if record:
                    hist[c].append(x.copy())
            X[:, c] = x
            its[c] = i
            states[c] = state
    if record:
        return X, its, states, hist
    return X, its


def dense_solve(A, b):
    """numpy LU solve of the dense matrix (tiny N only)."""
    Ad = A.toarray() if sp.issparse(A) else np.asarray(A, np.float64)
    return np.linalg.solve(Ad, np.asarray(b, np.float64))


def gauss_elim(A, b):
    """Gaussian elimination with partial pivoting, written out (tiny N only)."""
    M = (A.toarray() if sp.issparse(A) else np.array(A, np.float64)).copy()
    B = np.array(b, np.float64, copy=True)
    if B.ndim == 1:
        B = B[:, None]
    n = M.shape[0]
    for j in range(n):
        piv = j + int(np.argmax(np.abs(M[j:, j])))
        if piv != j:
            M[[j, piv]] = M[[piv, j]]
            B[[j, piv]] = B[[piv, j]]
        for i in range(j + 1, n):
            f = M[i, j] / M[j, j]
            if f != 0.0:
                M[i, j:] -= f * M[j, j:]
                B[i] -= f * B[j]
    X = np.zeros_like(B)
    for i in range(n - 1, -1, -1):
        X[i] = (B[i] - M[i, i + 1:] @ X[i + 1:]) / M[i, i]
    return X


def reference_solution(A, b, x0=None, rtol=1e-13, maxit=20000, stats=None):
    """x = A^{-1} b to a float64 true relative residual of about rtol.

    Textbook BiCGSTAB with Jacobi scaling, restarted from the true residual until
    ||b - A x|| / ||b|| <= rtol (joint over components).  ``stats`` (a dict, optional)
    receives the restarts and the BiCGSTAB iterations per component.
    """
    A = sp.csr_matrix(A, dtype=np.float64)
    b = np.asarray(b, np.float64)
    x = np.zeros_like(b) if x0 is None else np.asarray(x0, np.float64).copy()
    nb = np.linalg.norm(b)
    its_total = np.zeros(b.shape[1] if b.ndim > 1 else 1, np.int64)
    passes = 0
    for _ in range(20):
        r = b - A @ x
        if np.linalg.norm(r) <= rtol * nb:
            break
        d, its = bicgstab_textbook(A, r, None, eps=rtol * 0.1, maxit=maxit, jacobi=True)
        its_total += its
        passes += 1
        x = x + d
    if stats is not None:
        stats["passes"] = passes
        stats["iterations"] = [int(v) for v in its_total]
    return x
