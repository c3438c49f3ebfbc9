"""Kaiser-Bessel window of the NFFT, FP64. Test infrastructure only.

The paper leaves the NFFT window, the oversampling factor and the cutoff open
("controlled by several parameters, which we do not further discuss", Sec. 3.1)
and points to the NFFT literature (Plonka, Potts, Steidl, Tasche). The reading
taken here is the Kaiser-Bessel window with oversampling sigma = 2 and cutoff m:

    phi(x) = sinh(b sqrt(m^2 - (n x)^2)) / (pi sqrt(m^2 - (n x)^2)),   |x| <= m/n,
    b = pi (2 - 1/sigma),  n = sigma M.

Its Fourier transform phi_hat(k) = int phi(x) exp(-2 pi i k x) dx is computed
here by Gauss-Legendre quadrature of that definition (the integrand is an entire
function of x, so the quadrature converges fast). The published closed form
phi_hat(k) = I_0(m sqrt(b^2 - (2 pi k / n)^2)) / n is kept separately, as a pin.
"""
from __future__ import annotations

import numpy as np


def shape(sigma: float) -> float:
    return np.pi * (2.0 - 1.0 / sigma)


def phi(x, n: int, m: int, sigma: float = 2.0):
    """phi(x), x in physical units (the window has support |x| <= m/n)."""
    b = shape(sigma)
    t = np.asarray(x, dtype=np.float64) * n
    s2 = m * m - t * t
    out = np.zeros_like(t)
    inside = s2 >= 0
    s = np.sqrt(np.where(inside, s2, 0.0))
    small = inside & (s < 1e-8)
    big = inside & ~small
    out[big] = np.sinh(b * s[big]) / (np.pi * s[big])
    out[small] = b / np.pi
    return out


def phihat_quadrature(k, n: int, m: int, sigma: float = 2.0, nodes: int = 400):
    """phi_hat(k) = int_{-m/n}^{m/n} phi(x) cos(2 pi k x) dx (phi is even, so the sine part vanishes)."""
    z, w = np.polynomial.legendre.leggauss(nodes)
    x = z * (m / n)
    wx = w * (m / n)
    k = np.atleast_1d(np.asarray(k, dtype=np.float64))
    vals = phi(x, n, m, sigma)
    return (np.cos(2.0 * np.pi * np.outer(k, x)) * (vals * wx)[None, :]).sum(axis=1)


def phihat_closed_form(k, n: int, m: int, sigma: float = 2.0):
    """Published closed form, valid while |2 pi k / n| <= b."""
    b = shape(sigma)
    k = np.atleast_1d(np.asarray(k, dtype=np.float64))
    arg = b * b - (2.0 * np.pi * k / n) ** 2
    if np.any(arg < 0):
        raise ValueError("closed form used outside |k| <= n (1 - 1/(2 sigma))")
    return np.i0(m * np.sqrt(arg)) / n
