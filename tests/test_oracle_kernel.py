"""Pins of the Wendland and truncated Gaussian kernels (paper Sec. 5.2) against closed forms."""
import numpy as np
from scipy import integrate

from oracle import kernel


def test_unit_integral():
    # a smoothing kernel has unit integral: 4 pi int_0^2 w(q) q^2 dq = 1
    val, err = integrate.quad(lambda q: 4 * np.pi * kernel.w(q) * q * q, 0.0, 2.0, epsabs=1e-14)
    assert abs(val - 1.0) < 1e-12


def test_unit_integral_scaled():
    # W(r, h) = w(r/h)/h^3 integrates to one for any h
    for h in (0.013, 0.5, 2.0):
        val, _ = integrate.quad(lambda r: 4 * np.pi * kernel.W(r, h) * r * r, 0.0, 2 * h, epsabs=1e-14)
        assert abs(val - 1.0) < 1e-10


def test_f_is_derivative_over_q():
    # F = (1/r) dW/dr  <=>  f(q) = w'(q) / q; central differences
    q = np.linspace(0.05, 1.95, 39)
    e = 1e-6
    dw = (kernel.w(q + e) - kernel.w(q - e)) / (2 * e)
    np.testing.assert_allclose(kernel.f(q), dw / q, rtol=1e-7, atol=1e-10)


def test_support_edges_and_sign():
    assert kernel.w(2.0) == 0.0 and kernel.f(2.0) == 0.0
    assert kernel.w(2.5) == 0.0 and kernel.f(2.5) == 0.0
    q = np.linspace(0, 1.999, 200)
    assert np.all(kernel.f(q) < 0.0) and np.all(kernel.w(q) > 0.0)


def test_second_moment_of_F():
    # integration by parts: int r.grad W dV = -3 int W dV = -3, and r.grad W = r^2 F;
    # this pins the h^5 scaling of F against the h^3 scaling of W
    for h in (0.013, 1.0):
        val, _ = integrate.quad(lambda r: 4 * np.pi * kernel.F(r, h) * r ** 4, 0.0, 2 * h, epsabs=1e-14)
        assert abs(val + 3.0) < 1e-9


# ---- truncated Gaussian of radius 3 ----

def test_gaussian_unit_integral_and_norm():
    """w_G makes the truncated Gaussian integrate to one; w_G itself against the
    integral written out (4 pi int_0^3 (e^{-q^2} - e^{-9}) q^2 dq) by quadrature."""
    val, _ = integrate.quad(lambda q: 4 * np.pi * kernel.w_gauss(q) * q * q, 0.0, 3.0, epsabs=1e-14)
    assert abs(val - 1.0) < 1e-12
    raw, _ = integrate.quad(lambda q: 4 * np.pi * (np.exp(-q * q) - np.exp(-9.0)) * q * q, 0.0, 3.0, epsabs=1e-14)
    assert abs(raw - kernel.gauss_norm()) < 1e-12
    for h in (0.013, 0.5):
        val, _ = integrate.quad(lambda r: 4 * np.pi * kernel.W(r, h, kernel.GAUSSIAN) * r * r, 0.0, 3 * h,
                                epsabs=1e-14)
        assert abs(val - 1.0) < 1e-10


def test_gaussian_f_is_derivative_over_q_and_printed_magnitude():
    q = np.linspace(0.05, 2.95, 59)
    e = 1e-6
    dw = (kernel.w_gauss(q + e) - kernel.w_gauss(q - e)) / (2 * e)
    np.testing.assert_allclose(kernel.f_gauss(q), dw / q, rtol=1e-7, atol=1e-10)
    # the paper prints f = 2 exp(-q^2) / w_G: the magnitude of w'/q
    np.testing.assert_allclose(np.abs(kernel.f_gauss(q)), 2 * np.exp(-q * q) / kernel.gauss_norm(), rtol=1e-15)


def test_gaussian_support_edges():
    assert kernel.w_gauss(3.0) == 0.0 and kernel.w_gauss(3.5) == 0.0 and kernel.f_gauss(3.5) == 0.0
    assert kernel.support(kernel.GAUSSIAN) == 3.0 and kernel.support(kernel.WENDLAND) == 2.0


def test_gaussian_second_moment_of_F():
    # r.grad W integrates to -3 for any kernel vanishing at its support edge
    for h in (0.013, 1.0):
        val, _ = integrate.quad(lambda r: 4 * np.pi * kernel.F(r, h, kernel.GAUSSIAN) * r ** 4, 0.0, 3 * h,
                                epsabs=1e-14)
        assert abs(val + 3.0) < 1e-9
