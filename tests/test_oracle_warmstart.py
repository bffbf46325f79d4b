"""Pins of the warm-start reference (oracle/warmstart.py): the dummy-wall closure
(Eq. dummyvel), the fluid-block symmetry the library relies on, and the residual
targets against finite differences of the residual loss in parameter space."""
import numpy as np
import pytest

import scenes
from oracle import features as ofeat, kernel as okern, mlp as omlp, neighbors as onb, operator as oop
from oracle import warmstart as ows


def _system(s):
    off, idx = onb.build(s.pos, s.lo, s.hi, s.periodic, s.h)
    return off, idx, oop.assemble(s, off, idx)


def _rough(s, seed):
    """A velocity with both smooth and particle-scale content (walls at their own velocity)."""
    rng = np.random.default_rng(seed)
    v = np.array(s.vel, np.float32, copy=True)
    fl = s.ptype == scenes.FLUID
    v[fl, :3] += (0.3 * rng.standard_normal((int(fl.sum()), 3))).astype(np.float32)
    return v


@pytest.mark.parametrize("boundary", [scenes.BC_DUMMY, scenes.BC_DYNAMIC])
def test_closure_zeroes_wall_rows_of_the_residual(boundary):
    s = scenes.lava_box(0, n=6, boundary=boundary)
    _, _, A = _system(s)
    v = _rough(s, 1)
    x0 = ows.start(A, s.b, v, None, s.ptype, ows.fluid_scale(v, s.ptype))
    r = s.b - A @ x0
    wall = s.ptype != scenes.FLUID
    assert np.abs(r[wall]).max() <= 1e-14 * np.abs(x0).max()
    if boundary == scenes.BC_DYNAMIC:
        np.testing.assert_array_equal(x0[wall], s.b[wall])
    fl = ~wall
    np.testing.assert_array_equal(x0[fl], v[fl, :3].astype(np.float64))


def test_closure_is_the_shepard_formula():
    """x_w = b_w - sum_a W_wa x_a / sum_a W_wa over fluid neighbours a, from the kernel itself."""
    s = scenes.lava_box(1, n=5)
    off, idx, A = _system(s)
    v = _rough(s, 2)
    x0 = ows.start(A, s.b, v, None, s.ptype, 1.0)
    h = float(np.float32(s.h))
    P = np.asarray(s.pos, np.float32)[:, :3].astype(np.float64)
    checked = 0
    for w in np.flatnonzero(s.ptype != scenes.FLUID):
        nbrs = [a for a in idx[off[w]:off[w + 1]] if s.ptype[a] == scenes.FLUID and a != w]
        if not nbrs:
            np.testing.assert_array_equal(x0[w], s.b[w])       # empty Shepard sum: identity row
            continue
        Wt = np.array([okern.W(np.linalg.norm(P[a] - P[w]), h) for a in nbrs])
        ref = s.b[w] - (Wt[:, None] * v[nbrs, :3].astype(np.float64)).sum(0) / Wt.sum()
        np.testing.assert_allclose(x0[w], ref, rtol=1e-12, atol=1e-14)
        checked += 1
    assert checked > 50


@pytest.mark.parametrize("make", [lambda: scenes.lava_box(2, n=6),
                                  lambda: scenes.slope_subset(0, nx=8, ny=6, nz=8)])
def test_fluid_block_is_symmetric(make):
    """Equal masses and a symmetric viscosity mean give A_ff = A_ff^T, so A^T z = A z on
    fluid rows when z vanishes on wall rows (the library's shortcut for the gradient)."""
    s = make()
    _, _, A = _system(s)
    fl = np.flatnonzero(s.ptype == scenes.FLUID)
    Aff = A[fl][:, fl]
    assert abs(Aff - Aff.T).max() <= 1e-14 * abs(Aff).max()
    z = np.zeros((s.n, 3))
    z[fl] = np.random.default_rng(0).standard_normal((len(fl), 3))
    np.testing.assert_allclose((A.T @ z)[fl], (A @ z)[fl], rtol=0, atol=1e-12 * np.abs(A @ z).max())


def _net(seed):
    rng = np.random.default_rng(seed)
    p = omlp.init_params(seed)
    p["W4"] = p["W4"] * 5.0
    for k in ("b1", "b2", "b3", "b4"):
        p[k] = rng.normal(scale=0.05, size=p[k].shape)
    return p


@pytest.mark.parametrize("jacobi,log,highpass", [(True, True, False), (False, True, False), (True, False, False),
                                                  (False, False, False), (True, True, True), (False, False, True)])
def test_targets_give_the_loss_gradient(jacobi, log, highpass):
    """MSE gradient with the residual targets == central differences of L(theta) with the
    wall rows of x0 held at their closure values (FP64 network, no bf16 rounding)."""
    s = scenes.lava_box(3, n=5)
    off, idx, A = _system(s)
    v = _rough(s, 3)
    X, U = ofeat.features(s, off, idx, A, vel=v)
    fl = s.ptype == scenes.FLUID
    p = _net(4)
    y, _ = omlp.forward(p, X)
    S = ows.shepard_matrix(s, off, idx) if highpass else None
    t, x0, L = ows.residual_targets(A, s.b, v, y, s.ptype, U, jacobi, log, S)
    assert np.isfinite(L)
    _, g, _ = omlp.loss_and_grad(p, X, t, fl.astype(np.uint8))
    gflat = omlp.flatten(g)
    walls = x0[~fl].copy()

    def L_of(theta):
        yy, _ = omlp.forward(omlp.unflatten(theta), X)
        if S is not None:
            yy = yy - S @ yy
        x = x0.copy()
        x[fl] = v[fl, :3].astype(np.float64) + U * yy[fl]
        x[~fl] = walls
        return ows.loss(A, s.b, x, s.ptype, U, jacobi, log)

    assert abs(L_of(omlp.flatten(p)) - L) <= 1e-12 * max(1.0, abs(L))
    theta = omlp.flatten(p)
    rng = np.random.default_rng(5)
    eps = 1e-6
    for i in rng.choice(omlp.N_PARAMS, 12, replace=False):
        tp, tm = theta.copy(), theta.copy()
        tp[i] += eps
        tm[i] -= eps
        fd = (L_of(tp) - L_of(tm)) / (2 * eps)
        assert abs(fd - gflat[i]) <= 1e-5 * max(np.abs(gflat).max(), 1e-12), (i, fd, gflat[i])
    d = rng.standard_normal(omlp.N_PARAMS)
    d /= np.linalg.norm(d)
    fd = (L_of(theta + eps * d) - L_of(theta - eps * d)) / (2 * eps)
    assert abs(fd - gflat @ d) <= 1e-5 * abs(fd) + 1e-12, (fd, gflat @ d)


def test_log_loss_is_scale_free():
    """Scaling v, b (hence x*) by a constant leaves the log loss and the targets unchanged."""
    s = scenes.lava_box(4, n=5)
    off, idx, A = _system(s)
    v = _rough(s, 6)
    X, U = ofeat.features(s, off, idx, A, vel=v)
    y, _ = omlp.forward(_net(7), X)
    t1, _, L1 = ows.residual_targets(A, s.b, v, y, s.ptype, U)
    v2 = v.astype(np.float64) * 8.0
    t2, _, L2 = ows.residual_targets(A, 8.0 * s.b, v2, y, s.ptype, 8.0 * U)
    assert abs(L1 - L2) <= 1e-12 * abs(L1)
    np.testing.assert_allclose(t1, t2, rtol=1e-10, atol=1e-12)


def test_shepard_matrix_rows_and_constants():
    """S reproduces constants on fluid rows (rows sum to one), so (I - S) removes them;
    its weights are the kernel's, pinned against a direct sum for one row."""
    s = scenes.lava_box(5, n=5)
    off, idx, _ = _system(s)
    S = ows.shepard_matrix(s, off, idx)
    fl = s.ptype == scenes.FLUID
    np.testing.assert_allclose(np.asarray(S.sum(axis=1)).ravel()[fl], 1.0, rtol=1e-14)
    np.testing.assert_array_equal(np.asarray(S.sum(axis=1)).ravel()[~fl], 0.0)
    c = np.tile([0.3, -1.0, 2.0], (s.n, 1))
    np.testing.assert_allclose((c - S @ c)[fl], 0.0, atol=1e-14)
    b = int(np.flatnonzero(fl)[17])
    h = float(np.float32(s.h))
    P = np.asarray(s.pos, np.float32)[:, :3].astype(np.float64)
    V = np.asarray(s.pos, np.float32)[:, 3].astype(np.float64) / np.asarray(s.rho, np.float32).astype(np.float64)
    nb = [a for a in idx[off[b]:off[b + 1]] if fl[a]]
    w = {a: okern.W(np.linalg.norm(P[a] - P[b]), h) * V[a] for a in nb}
    w[b] = okern.W(0.0, h) * V[b]
    tot = sum(w.values())
    row = S.getrow(b).toarray().ravel()
    for a, wa in w.items():
        assert abs(row[a] - wa / tot) <= 1e-14
