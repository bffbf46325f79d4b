"""Neighbour sets of the SPH particles, in float64 (paper Sec. 5.2; reading X10).

Predicate (the definition both search routines below apply):
    alpha is a neighbour of beta  <=>  alpha != beta  and  r2 < (R h)^2
with R = 2 for the Wendland kernel and R = 3 for the truncated Gaussian (Sec. 5.2),
where, with the float32 inputs cast exactly to float64,
    d_a = x_alpha[a] - x_beta[a]                       for each axis a
    d_a = d_a - L_a * rint(d_a / L_a)                  on periodic axes (minimum image),
                                                       L_a = hi[a] - lo[a]
    r2  = (d_x*d_x + d_y*d_y) + d_z*d_z
    (R h)^2 = (R h) * (R h),  h = float64(h_float32)
Every operation is one IEEE float64 rounding in exactly this order, with no fused
multiply-add, so the set is reproducible bit for bit.  The kernels vanish at
q = R, so a strict inequality loses nothing (W = F = 0 there).

Output: CSR in caller order, ``offsets`` int64 [N+1], ``idx`` int32 [nnz], each row
ascending.
"""
import numpy as np

from . import kernel as _kernel


def _min_image(d, L):
    return d - L * np.rint(d / L)


def pair_r2(pos, a, b, lo, hi, periodic):
    """r2 for index arrays a (neighbour) and b (row), per the predicate above."""
    P = np.asarray(pos, dtype=np.float32)[:, :3].astype(np.float64)
    lo = np.asarray(lo, np.float64)
    hi = np.asarray(hi, np.float64)
    d = P[a] - P[b]
    for ax in range(3):
        if periodic[ax]:
            d[..., ax] = _min_image(d[..., ax], hi[ax] - lo[ax])
    return (d[..., 0] * d[..., 0] + d[..., 1] * d[..., 1]) + d[..., 2] * d[..., 2]


def support2(h, kernel_id=0):
    h2 = _kernel.support(kernel_id) * np.float64(np.float32(h))
    return h2 * h2


def bruteforce(pos, lo, hi, periodic, h, chunk=64, kernel_id=0):
    """All-pairs O(N^2) search: the definition of the neighbour sets."""
    P = np.asarray(pos, dtype=np.float32)[:, :3].astype(np.float64)
    n = P.shape[0]
    lo = np.asarray(lo, np.float64)
    hi = np.asarray(hi, np.float64)
    R2 = support2(h, kernel_id)
    rows = []
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        d = P[None, :, :] - P[s:e, None, :]          # [rows, N, 3]: x_alpha - x_beta
        for ax in range(3):
            if periodic[ax]:
                d[:, :, ax] = _min_image(d[:, :, ax], hi[ax] - lo[ax])
        r2 = (d[:, :, 0] * d[:, :, 0] + d[:, :, 1] * d[:, :, 1]) + d[:, :, 2] * d[:, :, 2]
        hit = r2 < R2
        hit[np.arange(e - s), np.arange(s, e)] = False
        for k in range(e - s):
            rows.append(np.flatnonzero(hit[k]).astype(np.int32))
    return _to_csr(rows, n)


def kdtree(pos, lo, hi, periodic, h, kernel_id=0):
    """k-d tree candidates (scipy, a library search) filtered by the exact predicate.

    The tree is queried with a slightly larger radius so that no pair that passes
    the float64 predicate can be missed by the tree's own rounding; the predicate
    then decides.  Equal to ``bruteforce`` on every scene (tests/test_oracle_neighbors.py).
    """
    from scipy.spatial import cKDTree

    P = np.asarray(pos, dtype=np.float32)[:, :3].astype(np.float64)
    n = P.shape[0]
    lo = np.asarray(lo, np.float64)
    hi = np.asarray(hi, np.float64)
    Q = P - lo
    box = np.empty(3)
    for ax in range(3):
        if periodic[ax]:
            L = hi[ax] - lo[ax]
            Q[:, ax] = np.mod(Q[:, ax], L)
            Q[Q[:, ax] >= L, ax] = 0.0
            box[ax] = L
        else:
            # an open axis: a period far larger than the extent
            box[ax] = 4.0 * (np.ptp(Q[:, ax]) + (hi[ax] - lo[ax]) + 1.0)
            Q[:, ax] -= Q[:, ax].min()
    tree = cKDTree(Q, boxsize=box)
    rad = _kernel.support(kernel_id) * float(np.float32(h)) * (1.0 + 1e-6)
    pairs = tree.query_pairs(rad, output_type="ndarray")
    a = np.concatenate([pairs[:, 0], pairs[:, 1]])
    b = np.concatenate([pairs[:, 1], pairs[:, 0]])
    r2 = pair_r2(pos, a, b, lo, hi, periodic)
    keep = r2 < support2(h, kernel_id)
    a, b = a[keep], b[keep]
    order = np.lexsort((a, b))
    a, b = a[order], b[order]
    offsets = np.zeros(n + 1, np.int64)
    np.add.at(offsets, b + 1, 1)
    offsets = np.cumsum(offsets)
    return offsets, a.astype(np.int32)


def build(pos, lo, hi, periodic, h, method="auto", kernel_id=0):
    n = np.asarray(pos).shape[0]
    if method == "bruteforce" or (method == "auto" and n <= 6000):
        return bruteforce(pos, lo, hi, periodic, h, kernel_id=kernel_id)
    return kdtree(pos, lo, hi, periodic, h, kernel_id=kernel_id)


def for_scene(scene, method="auto"):
    return build(scene.pos, scene.lo, scene.hi, scene.periodic, scene.h, method,
                 kernel_id=getattr(scene, "kernel", 0))


def rows_for(scene, rows):
    """Neighbour sets of a few rows by direct O(N) scans (for sampled checks at full size)."""
    n = scene.n
    out = []
    R2 = support2(scene.h, getattr(scene, "kernel", 0))
    allidx = np.arange(n)
    for b in np.asarray(rows, dtype=np.int64):
        r2 = pair_r2(scene.pos, allidx, np.full(n, b), scene.lo, scene.hi, scene.periodic)
        hit = r2 < R2
        hit[b] = False
        out.append(np.flatnonzero(hit).astype(np.int32))
    return out


def _to_csr(rows, n):
    offsets = np.zeros(n + 1, np.int64)
    offsets[1:] = np.cumsum([len(r) for r in rows])
    idx = np.concatenate(rows) if rows else np.zeros(0, np.int32)
    return offsets, idx.astype(np.int32)
