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


def test_bingham_slab_reaches_the_analytic_steady_profile():
    """A Papanastasiou slab driven by a body force g along x on a dummy-wall floor, periodic
    in x and z with a free top, marched with lagged viscosity (Sec. 3.3) and the implicit
    viscous system until it stops changing.  The steady state of a Bingham fluid is known in
    closed form: with the wall plane at y = 0, depth H and y_p = H - tau0 / (rho g),
    u = (rho g / mu0) (y_p y - y^2 / 2) below y_p and a rigid plug at (rho g / mu0) y_p^2 / 2
    above.  This pins the mu pass (velocity gradient, the D = sqrt(2 gdot:gdot) convention of
    reading X4, the regularised viscosity) together with the operator and the dummy walls:
    with D = sqrt(gdot:gdot) the same march yields a plug 37% slower."""
    from oracle import operator as oop
    import scipy.sparse.linalg as spla

    dx, ny, tau0, mu0, m, rho0, g, dt = 0.01, 30, 100.0, 10.0, 1000.0, 1000.0, 1.0, 5.0
    s = scenes.slope(0, nx=8, ny=ny, nz=8, dx=dx, rho0=rho0, tau0=tau0, mu0=mu0, m_reg=m, dt=dt,
                     noise=0.0, jitter=0.0)
    off, idx = neighbors.build(s.pos, s.lo, s.hi, s.periodic, s.h)
    nf = s.n_fluid
    y = s.pos[:nf, 1].astype(np.float64)
    yp = ny * dx - tau0 / (rho0 * g)
    ua = np.where(y <= yp, rho0 * g / mu0 * (yp * y - 0.5 * y * y), rho0 * g / mu0 * 0.5 * yp * yp)
    v = np.zeros((s.n, 4), np.float32)
    v[:nf, 0] = ua                       # the march's fixed point does not depend on the start
    for _ in range(200):
        mu, _ = rheology.mu_pass(s, off, idx, v)
        A = oop.assemble(s, off, idx, dt=dt, mu=mu)
        b = np.zeros((s.n, 3))
        b[:nf] = v[:nf, :3]
        b[:nf, 0] += dt * g
        x = spla.splu(A.tocsc()).solve(b)
        change = np.max(np.abs(x[:nf] - v[:nf, :3]))
        v[:, :3] = x.astype(np.float32)
        if change < 1e-6:
            break
    assert change < 1e-6
    u = x[:nf, 0]
    u_plug = rho0 * g / mu0 * 0.5 * yp * yp
    assert np.max(np.abs(u - ua)) <= 0.02 * u_plug
    plug = y > yp + 2 * s.h
    assert abs(u[plug].mean() - u_plug) <= 0.02 * u_plug
    assert np.std(u[plug]) <= 1e-3 * u_plug                # rigid
    np.testing.assert_array_equal(x[:nf, 1:], 0.0)       # no cross-flow from a pure shear
