"""Gradients of f = w^T K(theta) v, FP64. Test infrastructure only.

Parameters theta: the points x, each length scale ell_s, sigma_f, and v itself.

direct_grad   from the kernel's definition (Sec. 3.3):
                df/dv          = K w        (K is symmetric)
                df/d ell_s     = w^T (dK/d ell_s) v
                df/d sigma_f   = (2/sigma_f) w^T K v
                df/dx_{k,f}    = sigma_f^2 sum_s sum_j (w_k v_j + w_j v_k) d kappa_s(x_k - x_j)/d x_{k,f}
nfft_grad     the same derivatives of the NFFT approximation f~ = w^T K~ v (Sec. 3.1): with
              K~_s = A_s B_s A_s^T (A_s the interpolation matrix of window s, B_s symmetric), moving x_k
              changes row k of A_s, so
                df~/dx_k = sigma_f^2 sum_s [ w_k grad(A_s h_s(v))_k + v_k grad(A_s h_s(w))_k ]
              where h_s(u) = B_s A_s^T u is the interpolation grid of u and grad differentiates the
              window of the interpolation.
"""
from __future__ import annotations

import numpy as np

from . import _clib, fastsum, window


def direct_grad(points, windows, ell, sigma_f, v, w, rows=None):
    """Returns (grad_v, grad_ell[P], grad_sigma_f, grad_x[rows, d]) from the direct sums."""
    X = np.ascontiguousarray(points, dtype=np.float32)
    N, d = X.shape
    v = np.ascontiguousarray(v, dtype=np.float64)
    w = np.ascontiguousarray(w, dtype=np.float64)
    Kw, _ = fastsum.direct(X, windows, ell, sigma_f, w)
    Kv, dKv = fastsum.direct(X, windows, ell, sigma_f, v)
    rows = np.arange(N, dtype=np.int64) if rows is None else np.ascontiguousarray(rows, dtype=np.int64)
    off, feat = fastsum._csr(windows)
    ellc = np.ascontiguousarray(ell, dtype=np.float64)
    gx = np.zeros((len(rows), d))
    _clib.lib().orc_direct_grad_x(N, d, _clib.ptr(X), len(windows), _clib.ptr(off), _clib.ptr(feat),
                                  _clib.ptr(ellc), float(sigma_f), _clib.ptr(v), _clib.ptr(w), len(rows),
                                  _clib.ptr(rows), _clib.ptr(gx))
    return Kw, dKv @ w, 2.0 / sigma_f * (w @ Kv), gx


def _grid(x, u, chat, n, m, sigma):
    """Interpolation grid h(u) = B A^T u of one window (real, n^D), the same steps as nfft_fastsum."""
    M = chat.shape[0]
    d = x.shape[1]
    S = fastsum.nfft_adjoint(x, u, M, n, m, sigma)
    sl = tuple([slice(n // 2 - M // 2, n // 2 + M // 2)] * d)
    ghat = np.zeros((n,) * d, dtype=np.complex128)
    ghat[sl] = chat * S / (n ** d * fastsum._phihat_grid(M, n, m, sigma, d))
    return np.ascontiguousarray((np.fft.fftshift(np.fft.ifftn(np.fft.ifftshift(ghat))) * n ** d).real)


def gather_grad(x, h, n, m, sigma=2.0):
    """(values, gradients) of the interpolation sum_l h_l prod_t phi~(x_t - l_t/n) at the points x."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    N, d = x.shape
    val = np.zeros(N)
    grad = np.zeros((N, d))
    _clib.lib().orc_gather_grad(N, d, _clib.ptr(x), n, m, window.shape(sigma), _clib.ptr(h), _clib.ptr(val),
                                _clib.ptr(grad))
    return val, grad


def nfft_grad(points, windows, ell, sigma_f, v, w, bandwidth, cutoff, p=None, eps_B=1.0 / 16.0, sigma=2.0,
              reg=None):
    """Returns (grad_v, grad_ell[P], grad_sigma_f, grad_x[N, d]) of f~ = w^T K~ v. The coefficients
    (fastsum.coefficients_for) are held fixed in the coordinate gradient: under the separable reading
    their fit intervals are set-up constants of the operator, like the grid and the window."""
    X = np.asarray(points, dtype=np.float32).astype(np.float64)
    N, d = X.shape
    v = np.asarray(v, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    P = len(windows)
    if np.isscalar(bandwidth):
        bandwidth = [int(bandwidth)] * P
    Kw, dKw = fastsum.matvec_all(points, windows, ell, sigma_f, w, bandwidth, cutoff, p=p, eps_B=eps_B, sigma=sigma,
                                 reg=reg)
    Kv, _ = fastsum.matvec_all(points, windows, ell, sigma_f, v, bandwidth, cutoff, p=p, eps_B=eps_B, sigma=sigma,
                               reg=reg)
    gx = np.zeros((N, d))
    for s, win in enumerate(windows):
        M = int(bandwidth[s])
        n = int(round(sigma * M))
        xs = np.ascontiguousarray(X[:, list(win)])
        cg, _, _ = fastsum.coefficients_for(xs, float(ell[s]), M, p, eps_B, "gauss", reg)
        _, gv = gather_grad(xs, _grid(xs, v, cg, n, cutoff, sigma), n, cutoff, sigma)
        _, gw = gather_grad(xs, _grid(xs, w, cg, n, cutoff, sigma), n, cutoff, sigma)
        gx[:, list(win)] += sigma_f ** 2 * (w[:, None] * gv + v[:, None] * gw)
    return Kw, dKw @ v, 2.0 / sigma_f * (w @ Kv), gx
