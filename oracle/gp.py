"""Kernel ridge regression / GP training quantities in FP64. Test infrastructure only.

Sec. 3.3: the regression system (K + beta I) x = y (eq. "regression_system"), which the paper solves
with unpreconditioned conjugate gradients (Fig. "cg_iters_eigs": relative residual tolerance), and the
derivatives of K with respect to the hyperparameters that hyperparameter training needs:
    dK/d sigma_f = (2/sigma_f) K,   dK/d ell_s = sigma_f^2 (2/ell_s) K_s^der,   d(K + beta I)/d beta = I.

The paper motivates the derivative products with the gradient of a GP objective (Sec. 1: the
log-determinant term needs products with the derivative matrix). With A = K + beta I and
alpha = A^{-1} y, the Gaussian log marginal likelihood and its gradient are the textbook
    L(theta)     = -1/2 y^T alpha - 1/2 log det A - N/2 log(2 pi),
    dL/dtheta    =  1/2 alpha^T (dA/dtheta) alpha - 1/2 tr(A^{-1} dA/dtheta),
and Hutchinson's estimator replaces the trace by (1/m) sum_i (A^{-1} z_i)^T (dA/dtheta) z_i for
probe vectors z_i (given as input, e.g. Rademacher). Gradient order everywhere: (ell_1 .. ell_P,
sigma_f, beta).
"""
from __future__ import annotations

import numpy as np


def dense_kernel(points, windows, ell, sigma_f):
    """K and dK/d ell_s as dense FP64 matrices (Sec. 3.3 definitions):
        K_ij          = sigma_f^2 sum_s exp(-r_s^2 / (2 ell_s^2)),
        (dK/d ell_s)_ij = sigma_f^2 r_s^2 / ell_s^3 exp(-r_s^2 / (2 ell_s^2)),  r_s = ||x_i^W_s - x_j^W_s||."""
    X = np.asarray(points, dtype=np.float64)
    N = X.shape[0]
    K = np.zeros((N, N))
    dK = np.zeros((len(windows), N, N))
    for s, w in enumerate(windows):
        Y = X[:, list(w)]
        r2 = np.sum((Y[:, None, :] - Y[None, :, :]) ** 2, axis=2)
        E = np.exp(-r2 / (2.0 * ell[s] ** 2))
        K += sigma_f ** 2 * E
        dK[s] = sigma_f ** 2 * r2 / ell[s] ** 3 * E
    return K, dK


def cg(apply_A, Y, tol: float, maxit: int):
    """Conjugate gradients for A X = Y, every column on its own (A symmetric positive definite),
    started at X = 0; a column stops once ||r|| <= tol ||y||. Returns (X, iterations, relative
    residuals), iterations and residuals per column."""
    Y = np.asarray(Y, dtype=np.float64)
    one = Y.ndim == 1
    Y = Y.reshape(Y.shape[0], -1)
    X = np.zeros_like(Y)
    R = Y.copy()
    Pd = R.copy()
    rr = np.sum(R * R, axis=0)
    ynorm = np.sqrt(np.sum(Y * Y, axis=0))
    active = np.sqrt(rr) > tol * ynorm
    iters = np.zeros(Y.shape[1], dtype=np.int64)
    for _ in range(maxit):
        if not active.any():
            break
        AP = apply_A(Pd)
        pAp = np.sum(Pd * AP, axis=0)
        a = np.where(active, rr / np.where(active, pAp, 1.0), 0.0)
        X += a * Pd
        R -= a * AP
        rr_new = np.sum(R * R, axis=0)
        iters += active
        b = np.where(active, rr_new / np.where(active, rr, 1.0), 0.0)
        Pd = np.where(active, R + b * Pd, Pd)
        rr = np.where(active, rr_new, rr)
        active = active & (np.sqrt(rr) > tol * ynorm)
    rel = np.sqrt(rr) / ynorm
    if one:
        return X[:, 0], int(iters[0]), float(rel[0])
    return X, iters, rel


def lml(K, beta: float, y):
    """Log marginal likelihood of y under N(0, K + beta I), by a Cholesky factorisation."""
    y = np.asarray(y, dtype=np.float64)
    A = K + beta * np.eye(K.shape[0])
    Lc = np.linalg.cholesky(A)
    alpha = np.linalg.solve(Lc.T, np.linalg.solve(Lc, y))
    return -0.5 * y @ alpha - np.sum(np.log(np.diag(Lc))) - 0.5 * len(y) * np.log(2.0 * np.pi)


def _derivatives(K, dK, sigma_f):
    """dA/dtheta for theta = (ell_1 .. ell_P, sigma_f, beta) as a list of dense matrices."""
    return [dK[s] for s in range(dK.shape[0])] + [(2.0 / sigma_f) * K, np.eye(K.shape[0])]


def lml_grad_exact(K, dK, sigma_f: float, beta: float, y):
    """dL/dtheta with alpha and the traces computed exactly (dense solves)."""
    y = np.asarray(y, dtype=np.float64)
    A = K + beta * np.eye(K.shape[0])
    Ainv = np.linalg.inv(A)
    alpha = Ainv @ y
    return np.array([0.5 * alpha @ (D @ alpha) - 0.5 * np.sum(Ainv * D.T) for D in _derivatives(K, dK, sigma_f)])


def lml_grad_hutchinson_dense(K, dK, sigma_f: float, beta: float, y, Z):
    """dL/dtheta with the trace by Hutchinson's estimator over the probes Z (N x m) and dense solves:
    the exact value of the estimator the GPU path computes (which solves with CG)."""
    y = np.asarray(y, dtype=np.float64)
    Z = np.asarray(Z, dtype=np.float64).reshape(len(y), -1)
    A = K + beta * np.eye(K.shape[0])
    alpha = np.linalg.solve(A, y)
    W = np.linalg.solve(A, Z)
    m = Z.shape[1]
    return np.array([0.5 * alpha @ (D @ alpha) - 0.5 * np.sum(W * (D @ Z)) / m for D in _derivatives(K, dK, sigma_f)])


def lml_grad_hutchinson(apply_all, sigma_f: float, beta: float, y, Z, tol: float, maxit: int):
    """The same estimator through products only, as a fast-summation user runs it: apply_all(V)
    returns (K V, [dK/d ell_s V]) for the columns of V; the solves use cg on A = K + beta I.
    Returns (gradient, alpha, CG iterations)."""
    y = np.asarray(y, dtype=np.float64)
    Z = np.asarray(Z, dtype=np.float64).reshape(len(y), -1)
    m = Z.shape[1]
    B = np.column_stack([y, Z])
    S, iters, _ = cg(lambda V: apply_all(V)[0] + beta * V, B, tol, maxit)
    alpha, W = S[:, 0], S[:, 1:]
    KB, dKB = apply_all(np.column_stack([alpha, Z]))
    grad = []
    for s in range(len(dKB)):
        grad.append(0.5 * alpha @ dKB[s][:, 0] - 0.5 * np.sum(W * dKB[s][:, 1:]) / m)
    grad.append((2.0 / sigma_f) * (0.5 * alpha @ KB[:, 0] - 0.5 * np.sum(W * KB[:, 1:]) / m))
    grad.append(0.5 * alpha @ alpha - 0.5 * np.sum(W * Z) / m)
    return np.array(grad), alpha, iters


# --------------------------------------------------------------------- preconditioning ----
# Not in the paper (it solves with plain CG, tolerance 1e-3). At a small noise variance the system is
# ill-conditioned: for a kernel wide against the data, K = sigma_f^2 sum_s K_s has a few hundred large
# eigenvalues (about N times the leading Fourier coefficients) and the rest near zero, so
# kappa(K + beta I) ~ N / beta. The large eigenvalues belong to each window's lowest Fourier modes: in the
# fast summation K_s = sum_k c_hat_k e^{2 pi i k.(x - x')} (Sec. 3.1), and with the coefficients even,
# each pair +-k contributes 2 c_hat_k [cos(2 pi k.x) cos(2 pi k.x') + sin(2 pi k.x) sin(2 pi k.x')].
# The preconditioner keeps the modes with |k|_inf <= band of every window,
#     B = beta I + U W U^T,   U = [1, cos(2 pi k.x^{W_s}), sin(2 pi k.x^{W_s}) ...],
#     W = diag(sigma_f^2 sum_s c_hat_0^s, sigma_f^2 2 c_hat_k^s, ...),
# (the constant column shared by all windows), only modes with N sigma_f^2 2 c_hat_k >= beta (they lift
# an eigenvalue above the noise level), and applies B^{-1} by the Woodbury identity
#     B^{-1} r = (r - U (beta W^{-1} + U^T U)^{-1} U^T r) / beta.

def fourier_modes(windows, coefs, band: int, beta: float, sigma_f: float, N: int):
    """The retained modes: a list of (window s, k) and their weights, the constant mode first as
    (-1, None). coefs[s] is window s's c_hat array (shape (M,)*d_s, index k + M/2)."""
    import itertools
    modes, w = [(-1, None)], [sigma_f ** 2 * sum(float(c[tuple(n // 2 for n in c.shape)]) for c in coefs)]
    for s, c in enumerate(coefs):
        d, M = c.ndim, c.shape[0]
        for k in itertools.product(range(-band, band + 1), repeat=d):
            neg = tuple(-q for q in k)
            if k == (0,) * d or k < neg:                   # the zero mode is shared; one of each +-k pair
                continue
            val = 2.0 * sigma_f ** 2 * float(c[tuple(q + M // 2 for q in k)])
            if val > 0.0 and N * val >= beta:
                modes.append((s, k))
                w.append(val)
    return modes, np.array(w)


def fourier_basis(points, windows, modes) -> np.ndarray:
    """U (N x len(modes) columns, cosine and sine of each non-constant mode: 2 columns per mode but the
    constant's one). Returns U and the column weights' mode index per column."""
    X = np.asarray(points, dtype=np.float32).astype(np.float64)
    cols, owner = [], []
    for i, (s, k) in enumerate(modes):
        if s < 0:
            cols.append(np.ones(X.shape[0]))
            owner.append(i)
            continue
        ph = 2.0 * np.pi * (X[:, list(windows[s])] @ np.asarray(k, dtype=np.float64))
        cols += [np.cos(ph), np.sin(ph)]
        owner += [i, i]
    return np.column_stack(cols), np.asarray(owner)


def woodbury_apply(U, wcol, beta: float):
    """Returns a function r -> (beta I + U diag(wcol) U^T)^{-1} r by the Woodbury identity (FP64 Cholesky
    of beta diag(1/wcol) + U^T U)."""
    H = beta * np.diag(1.0 / wcol) + U.T @ U
    L = np.linalg.cholesky(H)

    def apply(r):
        r = np.asarray(r, dtype=np.float64)
        t = np.linalg.solve(L.T, np.linalg.solve(L, U.T @ r))
        return (r - U @ t) / beta
    return apply


def pcg(apply_A, apply_M, Y, tol: float, maxit: int):
    """Preconditioned conjugate gradients for A X = Y, every column on its own, from X = 0, with the
    flexible (Polak-Ribiere) direction update beta_k = r_{k+1}.(z_{k+1} - z_k) / r_k.z_k, which tolerates a
    preconditioner applied in FP32; a column stops once ||r|| <= tol ||y||. Returns (X, iterations, relative
    residuals of the recursion)."""
    Y = np.asarray(Y, dtype=np.float64)
    one = Y.ndim == 1
    Y = Y.reshape(Y.shape[0], -1)
    X = np.zeros_like(Y)
    R = Y.copy()
    Z = apply_M(R)
    Pd = Z.copy()
    rz = np.sum(R * Z, axis=0)
    ynorm = np.sqrt(np.sum(Y * Y, axis=0))
    active = np.sqrt(np.sum(R * R, axis=0)) > tol * ynorm
    iters = np.zeros(Y.shape[1], dtype=np.int64)
    for _ in range(maxit):
        if not active.any():
            break
        AP = apply_A(Pd)
        pAp = np.sum(Pd * AP, axis=0)
        a = np.where(active, rz / np.where(active, pAp, 1.0), 0.0)
        X = X + a * Pd
        R = R - a * AP                               # new arrays: apply_M may return its argument
        iters += active
        Zn = apply_M(R)
        b = np.where(active, np.sum(R * (Zn - Z), axis=0) / np.where(active, rz, 1.0), 0.0)
        Pd = np.where(active, Zn + b * Pd, Pd)
        rz = np.where(active, np.sum(R * Zn, axis=0), rz)
        Z = Zn
        active = active & (np.sqrt(np.sum(R * R, axis=0)) > tol * ynorm)
    rel = np.sqrt(np.sum(R * R, axis=0)) / ynorm
    if one:
        return X[:, 0], int(iters[0]), float(rel[0])
    return X, iters, rel
