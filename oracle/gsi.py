"""Global sensitivity indices of the fast-summation polynomial, FP64. Test infrastructure only.

Sec. 4 ("Global Sensitivity Analysis", Algorithm "Computation of GSI"): the approximation of
h(x) = sum_j v_j sum_s kappa_s(x_j^W_s, x^W_s) is, per window s, a trigonometric polynomial
    h~_s(x) = sum_{k in I_M^d_s} c_hat_k S(k, W_s) e^{...k.x},   S(k, W_s) = sum_j v_j e^{...k.x_j^W_s}
(the adjoint NFFT of v over the window's coordinates, step 2(a)). A frequency k whose non-zero
entries sit exactly on the positions of a subset u of the window's features contributes to the ANOVA
term of u (eq. "anova_fourier"), with variance |c_hat_k S(k, W_s)|^2 (step 2(b)). Summing those over
windows gives theta_u, over all non-empty u the total variance (step 3), and rho_u = theta_u / total
(step 4). Windows of any length d_s <= 3 and their own length scales are allowed (the paper's
"analogous" general case); subsets shared by several windows accumulate.

Reading: S uses the exponent sign of eq. "approx fast sum" (the adjoint NFFT,
S_k = sum_j v_j exp(-2 pi i k.x_j)), like every other product here; the paper's Sec. 4 writes the
opposite sign, which only relabels k -> -k.
"""
from __future__ import annotations

import itertools

import numpy as np

from . import fastsum


def window_spectrum(points, window, ell: float, v, M: int, p=None, eps_B: float = 1.0 / 16.0, reg=None):
    """c_hat_k S(k, W) for k in I_M^d (array indexed k + M/2), S by the exact trigonometric sum."""
    x = np.asarray(points, dtype=np.float32).astype(np.float64)[:, list(window)]
    chat, _, _ = fastsum.coefficients_for(x, float(ell), M, p, eps_B, "gauss", reg)
    S = fastsum.adjoint_exact(x, np.asarray(v, dtype=np.float64), M)
    return chat * S


def support_pattern(M: int, d: int) -> np.ndarray:
    """For every k in I_M^d (indexed k + M/2): the bit mask of its non-zero coordinates."""
    k = np.arange(-M // 2, M // 2)
    grids = np.meshgrid(*([k] * d), indexing="ij")
    pat = np.zeros((M,) * d, dtype=np.int64)
    for t in range(d):
        pat |= (grids[t] != 0).astype(np.int64) << t
    return pat


def gsi(points, windows, ell, v, bandwidth, p=None, eps_B: float = 1.0 / 16.0, reg=None):
    """Returns (rho, theta, total): dicts keyed by feature subsets (sorted tuples), rho_u = theta_u / total."""
    P = len(windows)
    if np.isscalar(bandwidth):
        bandwidth = [int(bandwidth)] * P
    theta = {}
    for s, w in enumerate(windows):
        M = int(bandwidth[s])
        spec = window_spectrum(points, w, ell[s], v, M, p, eps_B, reg)
        pat = support_pattern(M, len(w))
        e = np.abs(spec) ** 2
        for b in range(1, 2 ** len(w)):
            u = tuple(sorted(w[t] for t in range(len(w)) if b >> t & 1))
            theta[u] = theta.get(u, 0.0) + float(e[pat == b].sum())
    total = sum(theta.values())
    return {u: t / total for u, t in theta.items()}, theta, total


def subsets_of(windows):
    """Every non-empty subset of every window (sorted tuples), each once."""
    out = set()
    for w in windows:
        for r in range(1, len(w) + 1):
            for c in itertools.combinations(sorted(w), r):
                out.add(c)
    return sorted(out)
