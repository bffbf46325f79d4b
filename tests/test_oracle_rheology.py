"""Pins of the Papanastasiou viscosity pass (paper Sec. 2.1, 2.4) against closed forms."""
import itertools
import math

import numpy as np

import scenes
from oracle import kernel, neighbors, rheology


def _lattice_with_field(field, n=10):
    s = scenes.periodic_lattice(n)
    s.periodic = np.array([0, 0, 0], np.int32)   # open box so a linear field is admissible
    P = s.pos[:, :3].astype(np.float64)
    s.vel[:, :3] = field(P).astype(np.float32)
    off, idx = neighbors.build(s.pos, s.lo, s.hi, s.periodic, s.h)
    interior = np.all((P > 3 * s.dx) & (P < (n - 3) * s.dx), axis=1)
    return s, off, idx, interior


def _kappa(s):
    # lattice sum kappa = sum_delta V |F(|delta|)| delta_y^2 over the offsets inside 2h
    V = float(np.float32(s.pos[0, 3])) / float(np.float32(s.rho[0]))
    h = float(np.float32(s.h))
    k = 0.0
    for v in itertools.product(range(-3, 4), repeat=3):
        d = np.array(v, np.float64) * s.dx
        r = math.sqrt(d @ d)
        if v != (0, 0, 0) and r < 2 * h:
            k += V * abs(float(kernel.F(r, h))) * d[1] ** 2
    return k


def test_simple_shear_invariant_is_rate_times_lattice_sum():
    shear = 0.37
    s, off, idx, inner = _lattice_with_field(lambda P: np.stack([shear * P[:, 1], 0 * P[:, 0], 0 * P[:, 0]], 1))
    G = rheology.velocity_gradient(s, off, idx)
    D = rheology.shear_rate_invariant(G)
    kap = _kappa(s)
    assert abs(kap - 1.0) < 0.05         # the continuous moment int |F| r_y^2 dV = 1
    np.testing.assert_allclose(D[inner], shear * kap, rtol=2e-5)


def test_rigid_rotation_has_no_shear():
    om = np.array([0.3, -0.2, 0.5])
    s, off, idx, inner = _lattice_with_field(lambda P: np.cross(om, P - 0.05))
    D = rheology.shear_rate_invariant(rheology.velocity_gradient(s, off, idx))
    assert np.max(D[inner]) < 1e-5 * np.linalg.norm(om)


def test_papanastasiou_limits():
    tau0, mu0, m = 100.0, 1e3, 1000.0
    assert rheology.papanastasiou(0.0, tau0, mu0, m) == m * tau0 + mu0
    np.testing.assert_allclose(rheology.papanastasiou(1e-12, tau0, mu0, m), m * tau0 + mu0, rtol=1e-8)
    # large shear: the Bingham limit tau0 / D + mu0 (Eq. bingham)
    np.testing.assert_allclose(rheology.papanastasiou(10.0, tau0, mu0, m), tau0 / 10.0 + mu0, rtol=1e-12)


def test_series_truncation_bound():
    # alternating series: |T(x) - (1 - e^-x)/x| <= x^8 / 9!  for 0 <= x <= 1
    x = np.linspace(1e-6, 1.0, 200)
    exact = -np.expm1(-x) / x
    err = np.abs(rheology.series_T(x) - exact)
    assert np.all(err <= x ** 8 / math.factorial(9) * (1 + 1e-6) + 4e-16)
    # at the switch x0 = 0.5 the relative error is below single-precision epsilon
    assert abs(rheology.series_T(0.5) / (-math.expm1(-0.5) / 0.5) - 1) < 2 ** -24


def test_mu_pass_range_on_slope_subset():
    s = scenes.slope_subset(0, nx=12, ny=10, nz=12)
    off, idx = neighbors.build(s.pos, s.lo, s.hi, s.periodic, s.h)
    mu, D = rheology.mu_pass(s, off, idx)
    fl = s.ptype == scenes.FLUID
    tau0, mu0, m = s.rheology
    assert np.all(mu[fl] <= m * tau0 + mu0 + 1e-6) and np.all(mu[fl] > mu0)
