"""Smoothing kernels in float64 (paper Sec. 5.2, "Smoothing kernel choice").

Wendland psi_{3,1} (the default, support radius 2h): W(r, h) = w(r/h) / h^3 with
w(q) = 21/(16 pi) (1 - q/2)^4 (2q + 1) for q <= 2, and the gradient factor
F(r, h) = (1/r) dW/dr = f(r/h) / h^5 with f(q) = 105/(128 pi) (q - 2)^3
(Sec. 2.2 defines grad W = r F).  f <= 0 on [0, 2]: the kernel decreases.

Normalised truncated Gaussian of radius k = 3 (support radius 3h):
w(q) = (exp(-q^2) - exp(-k^2)) / w_G for q <= k, with
w_G = pi^(3/2) erf(k) - (2 pi / 3) exp(-k^2) k (3 + 2 k^2); its gradient factor
w'(q)/q = -2 exp(-q^2) / w_G (the paper prints the magnitude 2 exp(-q^2)/w_G; the
operator uses |F| either way, reading X1).

Pins (tests/test_oracle_kernel.py): 4 pi int w(q) q^2 dq = 1, f(q) = w'(q)/q,
w = f = 0 at and beyond the support, the second moment of F for both kernels.
"""
import math

import numpy as np

W_NORM = 21.0 / (16.0 * np.pi)
F_NORM = 105.0 / (128.0 * np.pi)

WENDLAND = 0
GAUSSIAN = 1
GAUSS_K = 3.0


def gauss_norm(k=GAUSS_K):
    """w_G, the normalisation of the truncated Gaussian (Sec. 5.2)."""
    return math.pi ** 1.5 * math.erf(k) - 2.0 * math.pi / 3.0 * math.exp(-k * k) * k * (3.0 + 2.0 * k * k)


def support(kernel_id=WENDLAND):
    """Support radius in units of h."""
    return GAUSS_K if kernel_id == GAUSSIAN else 2.0


def w_gauss(q):
    q = np.asarray(q, dtype=np.float64)
    return np.where(q <= GAUSS_K, (np.exp(-q * q) - math.exp(-GAUSS_K * GAUSS_K)) / gauss_norm(), 0.0)


def f_gauss(q):
    """w'(q)/q of the truncated Gaussian (negative inside the support)."""
    q = np.asarray(q, dtype=np.float64)
    return np.where(q <= GAUSS_K, -2.0 * np.exp(-q * q) / gauss_norm(), 0.0)


def w(q):
    """Dimensionless Wendland kernel w(q), zero beyond q = 2."""
    q = np.asarray(q, dtype=np.float64)
    t = 1.0 - 0.5 * q
    return np.where(q <= 2.0, W_NORM * t ** 4 * (2.0 * q + 1.0), 0.0)


def f(q):
    """Dimensionless gradient factor f(q) = w'(q)/q (negative inside the support)."""
    q = np.asarray(q, dtype=np.float64)
    return np.where(q <= 2.0, F_NORM * (q - 2.0) ** 3, 0.0)


def W(r, h, kernel_id=WENDLAND):
    """W(r, h) = w(r/h) / h^3."""
    h = float(h)
    ww = w_gauss if kernel_id == GAUSSIAN else w
    return ww(np.asarray(r, dtype=np.float64) / h) / h ** 3


def F(r, h, kernel_id=WENDLAND):
    """F(r, h) = f(r/h) / h^5, so that grad W(r) = r F(|r|)."""
    h = float(h)
    ff = f_gauss if kernel_id == GAUSSIAN else f
    return ff(np.asarray(r, dtype=np.float64) / h) / h ** 5
