"""Pins of the warm-start features (oracle/features.py) against closed forms on lattices."""
import itertools

import numpy as np
import pytest

import scenes
from oracle import features as ofeat, kernel, neighbors as onb, operator as oop


def _build(s):
    off, idx = onb.build(s.pos, s.lo, s.hi, s.periodic, s.h)
    return off, idx, oop.assemble(s, off, idx)


def _lattice_sums(s, kvec):
    """Direct sums over the integer lattice offsets inside 2h: the Fourier eigenvalue of A
    (1 + dt sum c (1 - cos k.d)), the diagonal D (1 + dt sum c), the Shepard sum
    (W(0) + sum W) V and the neighbour count."""
    dx, h = s.dx, float(np.float32(s.h))
    mu, m, rho = (float(np.float32(s.mu[0])), float(np.float32(s.pos[0, 3])), float(np.float32(s.rho[0])))
    lam, D, W, cnt = 1.0, 1.0, float(kernel.W(0.0, h)), 0
    for o in itertools.product(range(-3, 4), repeat=3):
        d = np.array(o, np.float64) * dx
        r = float(np.sqrt(d @ d))
        if o == (0, 0, 0) or r >= 2 * h:
            continue
        c = 2.0 * mu * m * abs(float(kernel.F(r, h))) / (rho * rho)
        lam += s.dt * c * (1.0 - np.cos(kvec @ d))
        D += s.dt * c
        W += float(kernel.W(r, h))
        cnt += 1
    return lam, D, W * m / rho, cnt


@pytest.mark.parametrize("modes", [(1, 0, 0), (0, 2, 1), (3, 3, 3)])
def test_neumann_features_on_a_fourier_mode(modes):
    """v = cos(k.r) e_x on the circulant lattice: e1 = (1 - lam) / D v and
    e2 = ((1 - lam) / D)^2 v exactly, D and lam from the lattice sums."""
    s = scenes.periodic_lattice(8, dt=3e-4)
    off, idx, A = _build(s)
    kvec = 2 * np.pi * np.array(modes) / (s.hi - s.lo)
    P = s.pos[:, :3].astype(np.float64)
    v = np.zeros((s.n, 4), np.float32)
    v[:, 0] = np.cos(P @ kvec)
    F, U = ofeat.features(s, off, idx, A, vel=v)
    lam, D, shep, cnt = _lattice_sums(s, kvec)
    vv = v[:, 0].astype(np.float64)
    g = (1.0 - lam) / D
    # v is the float32 rounding of cos(k.r) (error 6e-8); D^-1 (I - A) maps that rounding
    # noise with gain up to 2, and the second application again: 8 float32 ulps of |v| = 1
    tol = 8 * 2.0 ** -24
    np.testing.assert_allclose(F[:, 3] * U, g * vv, rtol=0, atol=tol)
    np.testing.assert_allclose(F[:, 6] * U, g * g * vv, rtol=0, atol=tol)
    assert abs(g) > 0.1 and g * g > 100 * tol
    np.testing.assert_array_equal(F[:, [4, 5, 7, 8]], 0.0)
    # the lattice positions are float32 (pair distances off by ~1e-7 relative)
    np.testing.assert_allclose(F[:, 10], np.log10(D) / 4.0, rtol=1e-6)
    np.testing.assert_allclose(F[:, 12], shep, rtol=1e-6)
    np.testing.assert_array_equal(F[:, 13], cnt / 80.0)
    assert cnt == 80
    np.testing.assert_array_equal(F[:, 11], 1.0)       # no walls
    np.testing.assert_array_equal(F[:, 15], 0.0)
    assert abs(U - np.sqrt((vv ** 2).mean())) <= 1e-12 * U


def test_constant_field_has_no_increment_and_balanced_neighbourhood():
    """A(dt) 1 = 1 on fluid rows (rows sum to one), so e1 = e2 = 0; every neighbour has the
    same speed, so feature 14 = 1/2; v / U = the unit direction."""
    s = scenes.lava_box(0, n=6)
    off, idx, A = _build(s)
    v = np.zeros((s.n, 4), np.float32)
    v[:, :3] = (0.3, -0.4, 1.2)
    F, U = ofeat.features(s, off, idx, A, vel=v)
    fl = s.ptype == scenes.FLUID
    assert abs(U - 1.3) <= 1e-7
    np.testing.assert_allclose(F[:, 3:9], 0.0, atol=1e-12)
    np.testing.assert_allclose(F[:, 14], 0.5, rtol=1e-12)
    np.testing.assert_allclose(F[:, 0:3], np.tile(np.array([0.3, -0.4, 1.2], np.float32) / 1.3, (s.n, 1)),
                               rtol=1e-6)
    np.testing.assert_array_equal(F[:, 15], (~fl).astype(float))
    # fluid particles of the bottom layer sit one spacing above the floor's top layer,
    # each coordinate jittered by at most 0.1 dx: nearest wall in [0.8, 1.2] dx
    low = fl & (s.pos[:, 2] < s.dx)
    dw = F[low, 11] * 2 * float(np.float32(s.h))
    assert low.sum() == 36 and np.all(dw >= 0.8 * s.dx) and np.all(dw <= 1.2 * s.dx)


def test_velocity_features_are_scale_free():
    s = scenes.lava_box(1, n=5)
    off, idx, A = _build(s)
    F1, U1 = ofeat.features(s, off, idx, A)
    v2 = s.vel.astype(np.float64) * 16.0
    F2, U2 = ofeat.features(s, off, idx, A, vel=v2.astype(np.float32))
    assert abs(U2 - 16.0 * U1) <= 1e-12 * U2
    np.testing.assert_allclose(F2, F1, rtol=1e-6, atol=1e-12)


def test_wall_rows_carry_the_stiffness_of_their_fluid_neighbours():
    """Feature 10 of a wall row is log10 of the mean diagonal D of its fluid neighbours / 4.
    In a Couette channel on a lattice whose dummy walls continue the lattice, every fluid
    particle sees the full lattice neighbourhood, so every fluid D is the lattice sum
    1 + dt sum c; wall rows within 2h of the fluid then carry log10 of that same D / 4 and
    the deeper ones 0."""
    s = scenes.couette(0, noise=0.0)
    off, idx, A = _build(s)
    F, _ = ofeat.features(s, off, idx, A)
    _, D, _, _ = _lattice_sums(s, np.zeros(3))
    fl = s.ptype == scenes.FLUID
    np.testing.assert_allclose(A.diagonal()[fl], D, rtol=1e-6)
    np.testing.assert_allclose(F[fl, 10], np.log10(D) / 4.0, rtol=1e-6)
    k = np.diff(A.tocsr().indptr) - 1
    near = (~fl) & (k > 0)
    assert near.sum() > 0 and (~fl & (k == 0)).sum() > 0
    np.testing.assert_allclose(F[near, 10], np.log10(D) / 4.0, rtol=1e-6)
    np.testing.assert_array_equal(F[(~fl) & (k == 0), 10], 0.0)


@pytest.mark.parametrize("kern,tol", [(scenes.KERNEL_GAUSSIAN, 2e-4), (scenes.KERNEL_WENDLAND, 2e-2)])
def test_shepard_feature_is_a_partition_of_unity_on_a_lattice(kern, tol):
    """Feature 12 (W(0) V_b + sum W_ba V_a with the scene's own kernel) on a perfect periodic
    lattice is the lattice quadrature of the kernel's unit integral: 1 up to the
    quadrature error, at h = 1.3 dx about 1e-4 for the truncated Gaussian (a smooth
    Gaussian would sum to 1 within exp(-pi^2 h^2 / dx^2) ~ 1e-7, but the truncation at 3h
    leaves a slope jump of 6 e^-9 ~ 7e-4 at the support edge) and about 1% for the
    Wendland kernel; a Shepard sum written with the wrong kernel misses by far more."""
    s = scenes.periodic_lattice(12, kernel=kern)
    off, idx = onb.build(s.pos, s.lo, s.hi, s.periodic, s.h, kernel_id=kern)
    A = oop.assemble(s, off, idx)
    F, _ = ofeat.features(s, off, idx, A)
    np.testing.assert_allclose(F[:, 12], 1.0, rtol=0, atol=tol)
