"""Pins of the assembled viscous matrix (paper Sec. 3.2) against closed forms and invariants."""
import itertools

import numpy as np
import pytest

import scenes
from oracle import kernel, neighbors, operator, solvers


def _build(s):
    off, idx = neighbors.build(s.pos, s.lo, s.hi, s.periodic, s.h, kernel_id=s.kernel)
    return off, idx, operator.assemble(s, off, idx)


@pytest.mark.parametrize("boundary", [scenes.BC_DUMMY, scenes.BC_DYNAMIC])
def test_zero_action_on_constants(boundary):
    # the viscous term annihilates a constant field: A 1 = 1 on fluid rows; a dummy
    # wall row with fluid neighbours gives 1 + 1 = 2 (Shepard weights sum to one);
    # dynamic wall rows and empty dummy rows are identity rows
    s = scenes.couette(0, boundary=boundary)
    off, idx, A = _build(s)
    y = A @ np.ones(s.n)
    fl = s.ptype == scenes.FLUID
    D = A.diagonal()
    assert np.all(np.abs(y[fl] - 1.0) <= 1e-13 * D[fl])
    S = operator.shepard_sums(s, off, idx)
    wall = ~fl
    if boundary == scenes.BC_DUMMY:
        np.testing.assert_allclose(y[wall & (S > 0)], 2.0, rtol=1e-14)
        np.testing.assert_array_equal(y[wall & (S == 0)], 1.0)
    else:
        np.testing.assert_array_equal(y[wall], 1.0)


def test_zero_action_on_constants_gaussian():
    """The same invariant with the truncated Gaussian (support 3h) on a box with four
    dummy layers (the 3.9 dx support reaches the fourth layer)."""
    s = scenes.lava_box(1, n=8, layers=4, kernel=scenes.KERNEL_GAUSSIAN)
    off, idx, A = _build(s)
    assert np.diff(off)[s.ptype == scenes.FLUID].max() > 200
    y = A @ np.ones(s.n)
    fl = s.ptype == scenes.FLUID
    assert np.all(np.abs(y[fl] - 1.0) <= 1e-13 * A.diagonal()[fl])
    S = operator.shepard_sums(s, off, idx)
    np.testing.assert_allclose(y[~fl & (S > 0)], 2.0, rtol=1e-14)


def test_sdd_margin_is_one_and_wall_rows_wcdd():
    s = scenes.random_box(3, nf=300, mu_spread=9.0, mass_spread=0.5)
    off, idx, A = _build(s)
    Ad = A.toarray()
    off_abs = np.abs(Ad).sum(axis=1) - np.abs(np.diag(Ad))
    fl = s.ptype == scenes.FLUID
    # fluid rows: diag - sum|off| = 1 exactly in exact arithmetic (reading X1)
    np.testing.assert_allclose(np.diag(Ad)[fl] - off_abs[fl], 1.0, rtol=0, atol=1e-12 * np.diag(Ad).max())
    assert np.all(Ad[fl][:, :][~np.eye(s.n, dtype=bool)[fl]] <= 0.0)
    # dummy wall rows: |diag| = sum|off| = 1 (only weak dominance), off-diagonals
    # only towards fluid columns, which are SDD rows: WCDD
    S = operator.shepard_sums(s, off, idx)
    w = (~fl) & (S > 0)
    np.testing.assert_allclose(off_abs[w], 1.0, rtol=1e-14)
    cols = np.nonzero(Ad[w] - np.diag(np.diag(Ad))[w])[1]
    assert np.all(fl[cols])


@pytest.mark.parametrize("mean", [scenes.MEAN_HARMONIC, scenes.MEAN_ARITHMETIC])
def test_symmetric_without_walls(mean):
    # no walls, periodic, uniform mass and density: A = A^T bit for bit, with the
    # symmetric evaluation of App. A (r_ab computed as one difference)
    s = scenes.periodic_lattice(8, jitter=0.1, mu_spread=4.0, seed=2)
    s.mean = mean
    off, idx, A = _build(s)
    D = (A - A.T).tocoo()
    assert D.nnz == 0 or np.max(np.abs(D.data)) == 0.0


def test_not_symmetric_with_dummy_walls():
    s = scenes.couette(0)
    off, idx, A = _build(s)
    assert abs(A - A.T).max() > 0.1


def _stencil_eigenvalue(s, kvec):
    # lambda(k) = 1 + dt sum_{delta in stencil} c(|delta|) (1 - cos(k.delta)), with the
    # stencil the lattice offsets strictly inside 2h = 2.6 dx
    dx = s.dx
    lam = 1.0
    mu = float(np.float32(s.mu[0]))
    m = float(np.float32(s.pos[0, 3]))
    rho = float(np.float32(s.rho[0]))
    h = float(np.float32(s.h))
    R = kernel.support(s.kernel)
    for v in itertools.product(range(-4, 5), repeat=3):
        d = np.array(v, np.float64) * dx
        r = np.sqrt(d @ d)
        if v == (0, 0, 0) or r >= R * h:
            continue
        c = 2.0 * mu * m * abs(float(kernel.F(r, h, s.kernel))) / (rho * rho)
        lam += s.dt * c * (1.0 - np.cos(kvec @ d))
    return lam


@pytest.mark.parametrize("modes", [(1, 0, 0), (0, 2, 1), (3, 3, 3), (4, 0, 4), (1, 2, 3)])
@pytest.mark.parametrize("kern", [scenes.KERNEL_WENDLAND, scenes.KERNEL_GAUSSIAN])
def test_fourier_closed_form(modes, kern):
    # perfect periodic lattice, uniform mu/rho/m: the operator is circulant, so
    # A cos(k.r) = lambda(k) cos(k.r) with the stencil-sum eigenvalue (any kernel)
    s = scenes.periodic_lattice(8 if kern == scenes.KERNEL_WENDLAND else 12, dt=3e-4, kernel=kern)
    off, idx, A = _build(s)
    L = s.hi - s.lo
    kvec = 2 * np.pi * np.array(modes) / L
    P = s.pos[:, :3].astype(np.float64)
    v = np.cos(P @ kvec)
    lam = _stencil_eigenvalue(s, kvec)
    assert lam > 2.0 or modes == (1, 0, 0)
    np.testing.assert_allclose(A @ v, lam * v, rtol=0, atol=2e-6 * lam)
    # and the solve: x = b / lambda
    x = solvers.reference_solution(A, v[:, None])
    np.testing.assert_allclose(x[:, 0], v / lam, rtol=0, atol=2e-6)


def test_dynamic_walls_are_identity_rows_but_enter_fluid_rows():
    s = scenes.couette(0, boundary=scenes.BC_DYNAMIC)
    off, idx, A = _build(s)
    Ad = A.toarray()
    wall = s.ptype == scenes.WALL
    np.testing.assert_array_equal(Ad[wall], np.eye(s.n)[wall])
    fl_near = np.flatnonzero((s.ptype == scenes.FLUID) & (s.pos[:, 1] < 0.01))
    assert np.all((Ad[np.ix_(fl_near, np.flatnonzero(wall))] < 0).sum(axis=1) > 0)


def test_rows_apply_matches_assembled():
    s = scenes.random_box(4, nf=300, mu_spread=3.0)
    off, idx, A = _build(s)
    rng = np.random.default_rng(0)
    x = rng.normal(size=(s.n, 3))
    rows = [0, 5, 100, s.n - 1, s.n - 40]
    nb = [idx[off[b]:off[b + 1]] for b in rows]
    np.testing.assert_allclose(operator.rows_apply(s, rows, nb, x), (A @ x)[rows], rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("boundary", [scenes.BC_DUMMY, scenes.BC_DYNAMIC])
def test_row_norms_against_rowwise_sums_and_bounds(boundary):
    """row_norms2 against an explicit row-by-row sum of (A_ij / A_ii)^2, and the bounds
    the rows' structure fixes: a dummy-wall row with k fluid neighbours carries weights
    W / S that sum to one, so 1 + 1/k <= norm2 <= 2; dynamic and lone wall rows are
    identity rows (norm2 = 1); a fluid row's off-diagonal magnitudes sum to D - 1, so
    (D-1)^2 / (k D^2) <= norm2 - 1 <= (D-1)^2 / D^2 over its k neighbours."""
    s = scenes.couette(3, nx=8, ny=6, nz=8, boundary=boundary)
    off, idx = neighbors.build(s.pos, s.lo, s.hi, s.periodic, s.h)
    A = operator.assemble(s, off, idx).tocsr()
    rn2 = operator.row_norms2(A)
    for i in range(0, s.n, 7):
        lo, hi = A.indptr[i], A.indptr[i + 1]
        d = A[i, i]
        want = sum((A.data[j] / d) ** 2 for j in range(lo, hi))
        assert abs(rn2[i] - want) <= 1e-14 * want
    fl = s.ptype == scenes.FLUID
    k = np.diff(A.indptr) - 1                    # off-diagonal entries per row
    D = A.diagonal()
    f = fl & (k > 0)
    assert np.all(rn2[f] - 1 <= (D[f] - 1) ** 2 / D[f] ** 2 * (1 + 1e-12))
    assert np.all(rn2[f] - 1 >= (D[f] - 1) ** 2 / (k[f] * D[f] ** 2) * (1 - 1e-12))
    w = ~fl
    if boundary == scenes.BC_DYNAMIC:
        np.testing.assert_array_equal(rn2[w], 1.0)
    else:
        wk = w & (k > 0)
        assert wk.sum() > 0
        assert np.all(rn2[wk] <= 2.0 + 1e-12) and np.all(rn2[wk] >= 1.0 + 1.0 / k[wk] - 1e-12)
        np.testing.assert_array_equal(rn2[w & (k == 0)], 1.0)


def test_wall_row_scale_leaves_fluid_rows_and_falls_with_power():
    s = scenes.lava_box(2, n=8)
    off, idx = neighbors.build(s.pos, s.lo, s.hi, s.periodic, s.h)
    A = operator.assemble(s, off, idx)
    fl = s.ptype == scenes.FLUID
    s0 = operator.wall_row_scale(s, A, 0.0)
    s3 = operator.wall_row_scale(s, A, 3.0)
    s4 = operator.wall_row_scale(s, A, 4.0)
    np.testing.assert_array_equal(s0, 1.0)
    np.testing.assert_array_equal(s3[fl], 1.0)
    assert np.all(s4[~fl] <= s3[~fl]) and np.all(s3[~fl] <= 1.0) and np.all(s3[~fl] >= 0.125)
    assert np.any(s3[~fl] < 0.5)
    # a constant factor on the Shepard rows only: lone walls (identity rows) keep 1
    k = np.diff(A.tocsr().indptr) - 1
    c = operator.wall_row_scale(s, A, 0.0, factor=0.25)
    np.testing.assert_array_equal(c[fl], 1.0)
    np.testing.assert_array_equal(c[(~fl) & (k > 0)], 0.25)
    np.testing.assert_array_equal(c[(~fl) & (k == 0)], 1.0)
    assert ((~fl) & (k == 0)).sum() > 0
