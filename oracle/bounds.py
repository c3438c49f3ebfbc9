"""Error bounds of Sec. 3.4 and the analytic Fourier coefficients of Sec. 3.1, FP64.
Test infrastructure only.

Notation of the paper: M (the paper's m) Fourier coefficients per dimension,
eta = ell pi M / sqrt(2). Bounds hold for eta >= 1 and the plain periodic
continuation of the kernel on [-1/2,1/2]^d (no regularisation).

Reading: in Theorem "multi_gauss" the statement gives ell e^{-1/2}/eta^2 for the
ell >= 1/2 branch of gamma, while the proof derives 2 ell e^{-1/2}/eta^2. The
larger (proof) value is used, so the bound stays an upper bound.
"""
from __future__ import annotations

import numpy as np
from scipy.special import erfc, wofz

SQ2PI = np.sqrt(2.0 * np.pi)
ELL_STAR = 0.5 * np.sqrt(2.0 / (5.0 + np.sqrt(17.0)))    # case split of Theorem "multi_deriv"


def eta(ell: float, M: int) -> float:
    return ell * np.pi * M / np.sqrt(2.0)


def gamma(e: float, ell: float) -> float:
    """gamma(eta, ell) of Theorem "multi_gauss" (bound on |c_{M/2}(f)|)."""
    tail = np.exp(-1.0 / (8 * ell * ell)) / e ** 2 if ell < 0.5 else 2.0 * ell * np.exp(-0.5) / e ** 2
    return ell * SQ2PI * np.exp(-e * e) + tail


def A(e: float, ell: float) -> float:
    """A(eta, ell) of Theorem "multi_gauss" (bound on sum_{k > M/2} |c_k(f)|)."""
    tail = (np.exp(-1.0 / (8 * ell * ell)) / (np.sqrt(2.0) * ell * np.pi * e) if ell < 0.5
            else np.sqrt(2.0) * np.exp(-0.5) / (np.pi * e))
    return np.exp(-e * e) / (2.0 * e * np.sqrt(np.pi)) + tail


def xi(e: float, ell: float) -> float:
    """xi(eta, ell) of Theorem "multi_deriv" (bound on |c_{M/2}(g)|)."""
    tail = (np.exp(-1.0 / (8 * ell * ell)) / (8 * e * e * ell * ell) if ell <= ELL_STAR
            else 1.0 / e ** 2 + 3.0 * ell / (2.0 * e ** 2))
    return (e * e + 0.5) * ell * SQ2PI * np.exp(-e * e) + tail


def S(e: float, ell: float) -> float:
    """S(eta, ell) of Theorem "multi_deriv" (bound on sum_{k > M/2} |c_k(g)|)."""
    tail = (np.exp(-1.0 / (8 * ell * ell)) / (8 * np.sqrt(2.0) * np.pi * ell ** 3 * e) if ell <= ELL_STAR
            else 1.0 / (np.sqrt(2.0) * np.pi * ell * e) + 3.0 / (2.0 * np.sqrt(2.0) * np.pi * e))
    return (erfc(e) / 4.0 + e * np.exp(-e * e) / (2.0 * np.sqrt(np.pi))
            + np.exp(-e * e) / (4.0 * np.sqrt(np.pi) * e) + tail)


def bound_gauss_3d(ell: float, M: int) -> float:
    """Theorem "multi_gauss": ||kappa_ERR||_inf <= 15 gamma (gamma + 5/2) + 102 A."""
    e = eta(ell, M)
    g = gamma(e, ell)
    return 15.0 * g * (g + 2.5) + 102.0 * A(e, ell)


def bound_der_3d(ell: float, M: int) -> float:
    """Theorem "multi_deriv": (5/2 xi + 15 gamma)(15 + 12 gamma) + 75 S + 6 A (116/5 S + 87)."""
    e = eta(ell, M)
    g, a, x, s = gamma(e, ell), A(e, ell), xi(e, ell), S(e, ell)
    return (2.5 * x + 15.0 * g) * (15.0 + 12.0 * g) + 75.0 * s + 6.0 * a * (116.0 / 5.0 * s + 87.0)


def bound_gauss_1d(ell: float, M: int) -> float:
    """Remark "gaussian1d": 2 gamma + 4 A."""
    e = eta(ell, M)
    return 2.0 * gamma(e, ell) + 4.0 * A(e, ell)


def bound_der_1d(ell: float, M: int) -> float:
    """Remark "deriv1d": 2 xi + 4 S."""
    e = eta(ell, M)
    return 2.0 * xi(e, ell) + 4.0 * S(e, ell)


def analytic_coeff_gauss_1d(k, ell: float):
    """c_k of the 1-periodic continuation of exp(-r^2/(2 ell^2)) from [-1/2,1/2] (Sec. 3.1):
        c_k = ell sqrt(2 pi) exp(-2 pi^2 k^2 ell^2) Re erf(1/(2 sqrt2 ell) + i pi k sqrt2 ell).
    Evaluated through the Faddeeva function to avoid overflow: with z = alpha + i beta,
    exp(-beta^2) erf(z) = exp(-beta^2) - exp(-alpha^2 - 2 i alpha beta) w(i z)."""
    k = np.asarray(k, dtype=np.float64)
    alpha = 1.0 / (2.0 * np.sqrt(2.0) * ell)
    beta = np.pi * k * np.sqrt(2.0) * ell
    iz = -beta + 1j * alpha
    val = np.exp(-beta ** 2) - np.exp(-alpha ** 2 - 2j * alpha * beta) * wofz(iz)
    return ell * SQ2PI * val.real
