"""Windows of the NFFT, FP64: Kaiser-Bessel (default) and exponential of semicircle. Test infrastructure only.

The paper leaves the NFFT window, the oversampling factor and the cutoff open
(Sec. 3.1 does not discuss the NFFT's accuracy parameters) and points to the NFFT
literature (Plonka, Potts, Steidl, Tasche). The reading
taken here is the Kaiser-Bessel window with oversampling sigma = 2 and cutoff m:

    phi(x) = sinh(b sqrt(m^2 - (n x)^2)) / (pi sqrt(m^2 - (n x)^2)),   |x| <= m/n,
    b = pi (2 - 1/sigma),  n = sigma M.

Its Fourier transform phi_hat(k) = int phi(x) exp(-2 pi i k x) dx is computed
here by Gauss-Legendre quadrature of that definition (the integrand is an entire
function of x, so the quadrature converges fast). The published closed form
phi_hat(k) = I_0(m sqrt(b^2 - (2 pi k / n)^2)) / n is kept separately, as a pin.

The exponential-of-semicircle window (Barnett, Magland, af Klinteberg, SIAM J. Sci. Comput. 2019)
is offered as the alternative the NFFT literature allows:

    phi(x) = exp(beta (sqrt(1 - (n x / m)^2) - 1)),   |x| <= m/n,

with beta = 2.30 * 2m at sigma = 2 (that paper's choice for upsampling 2), scaled by
(1 - 1/(2 sigma)) / (3/4) for other sigma. It has no closed-form transform; phi_hat comes from
the same quadrature (the square-root edge behaviour is weighted by exp(-beta)).
"""
from __future__ import annotations

import numpy as np


KINDS = {"kb": 0, "es": 1}


def shape(sigma: float) -> float:
    return np.pi * (2.0 - 1.0 / sigma)


def es_beta(m: int, sigma: float = 2.0) -> float:
    """Shape beta of the exponential-of-semicircle window with cutoff m (width 2m grid points)."""
    return 2.30 * 2 * m * (1.0 - 1.0 / (2.0 * sigma)) / 0.75


def shape_of(m: int, sigma: float = 2.0, window: str = "kb") -> float:
    """The shape parameter the spreading/interpolation code takes: b (Kaiser-Bessel) or beta (ES)."""
    return es_beta(m, sigma) if window == "es" else shape(sigma)


def phi(x, n: int, m: int, sigma: float = 2.0, window: str = "kb"):
    """phi(x), x in physical units (the window has support |x| <= m/n)."""
    if window == "es":
        beta = es_beta(m, sigma)
        z = np.asarray(x, dtype=np.float64) * (n / m)
        s2 = 1.0 - z * z
        out = np.zeros_like(z)
        inside = s2 >= 0
        out[inside] = np.exp(beta * (np.sqrt(s2[inside]) - 1.0))
        return out
    if window != "kb":
        raise ValueError(window)
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


def phihat_quadrature(k, n: int, m: int, sigma: float = 2.0, nodes: int = 400, window: str = "kb"):
    """phi_hat(k) = int_{-m/n}^{m/n} phi(x) cos(2 pi k x) dx (phi is even, so the sine part vanishes)."""
    z, w = np.polynomial.legendre.leggauss(nodes)
    x = z * (m / n)
    wx = w * (m / n)
    k = np.atleast_1d(np.asarray(k, dtype=np.float64))
    vals = phi(x, n, m, sigma, window)
    return (np.cos(2.0 * np.pi * np.outer(k, x)) * (vals * wx)[None, :]).sum(axis=1)


def phihat_closed_form(k, n: int, m: int, sigma: float = 2.0):
    """Published closed form, valid while |2 pi k / n| <= b."""
    b = shape(sigma)
    k = np.atleast_1d(np.asarray(k, dtype=np.float64))
    arg = b * b - (2.0 * np.pi * k / n) ** 2
    if np.any(arg < 0):
        raise ValueError("closed form used outside |k| <= n (1 - 1/(2 sigma))")
    return np.i0(m * np.sqrt(arg)) / n
