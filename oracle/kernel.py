"""Wendland psi_{3,1} smoothing kernel in float64 (paper Sec. 5.2, "Smoothing kernel choice").

W(r, h) = w(r/h) / h^3 with w(q) = 21/(16 pi) (1 - q/2)^4 (2q + 1) for q <= 2, and the
gradient factor F(r, h) = (1/r) dW/dr = f(r/h) / h^5 with f(q) = 105/(128 pi) (q - 2)^3
(Sec. 2.2 defines grad W = r F).  f <= 0 on [0, 2]: the kernel decreases.

Pins (tests/test_oracle_kernel.py): 4 pi int_0^2 w(q) q^2 dq = 1, f(q) = w'(q)/q,
w(2) = f(2) = 0.
"""
import numpy as np

W_NORM = 21.0 / (16.0 * np.pi)
F_NORM = 105.0 / (128.0 * np.pi)


def w(q):
    """Dimensionless Wendland kernel w(q), zero beyond q = 2."""
    q = np.asarray(q, dtype=np.float64)
    t = 1.0 - 0.5 * q
    return np.where(q <= 2.0, W_NORM * t ** 4 * (2.0 * q + 1.0), 0.0)


def f(q):
    """Dimensionless gradient factor f(q) = w'(q)/q (negative inside the support)."""
    q = np.asarray(q, dtype=np.float64)
    return np.where(q <= 2.0, F_NORM * (q - 2.0) ** 3, 0.0)


def W(r, h):
    """W(r, h) = w(r/h) / h^3."""
    h = float(h)
    return w(np.asarray(r, dtype=np.float64) / h) / h ** 3


def F(r, h):
    """F(r, h) = f(r/h) / h^5, so that grad W(r) = r F(|r|)."""
    h = float(h)
    return f(np.asarray(r, dtype=np.float64) / h) / h ** 5
