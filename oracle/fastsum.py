"""Fast summation, FP64, three levels, plus the direct sums. Test infrastructure only.

Levels, as in the error decomposition of Sec. 3.4.4 (direct -> Fourier
approximation -> NFFT):

1. direct(...)      the plain definition of K v and dK/d ell_s v (Sec. 3.3).
2. ndft_fastsum     the trigonometric-polynomial sum of eq. "approx fast sum"
                    (Sec. 3.1), evaluated exactly (no window):
                        h~(x_i) = sum_k c_hat_k S_k exp(+2 pi i k.x_i),
                        S_k     = sum_j v_j exp(-2 pi i k.x_j).
3. nfft_fastsum     the same sum computed the way the paper describes it
                    (Sec. 3.1 and Sec. 3.4): the inner sums S_k by an adjoint
                    NFFT, the multiplication by c_hat_k, the outer sums by an
                    NFFT. Each NFFT is spreading/interpolation with the window
                    phi on the oversampled grid of n = sigma M points per
                    dimension, an n^d FFT, and division by phi_hat (the window's
                    Fourier transform), following the standard NFFT derivation:
                        adjoint: S_k ~= G_k / (n^d prod_t phi_hat(k_t)),
                                 G_k = sum_l g_l exp(-2 pi i k.l/n),
                                 g_l = sum_j v_j phi~(x_j - l/n);
                        forward: f(x) ~= sum_l h_l phi~(x - l/n),
                                 h_l = sum_{k in I_M} (d_k / (n^d prod_t phi_hat(k_t))) exp(+2 pi i k.l/n).

Additive kernel (Sec. 1 eq. "wind_gauss_anova_kernel", Sec. 3.3):
    K v          = sigma_f^2 sum_s K_s^gauss v
    dK/d ell_s v = sigma_f^2 (2/ell_s) K_s^der v
    dK/d sigma_f v = (2/sigma_f) K v
"""
from __future__ import annotations

import functools

import numpy as np

from . import _clib
from . import kernels
from . import window


def _csr(windows):
    off = [0]
    feat = []
    for w in windows:
        feat.extend(int(f) for f in w)
        off.append(len(feat))
    return np.asarray(off, dtype=np.int32), np.asarray(feat, dtype=np.int32)


def direct(points: np.ndarray, windows, ell, sigma_f: float, v: np.ndarray, rows=None):
    """Direct FP64 sums for the rows `rows` (all rows if None).

    Returns (Kv[rows], dK[P, rows]) with
        (K v)_i          = sigma_f^2 sum_s sum_j exp(-||x_i^W_s - x_j^W_s||^2 / (2 ell_s^2)) v_j
        (dK/d ell_s v)_i = sigma_f^2 sum_j ||x_i^W_s - x_j^W_s||^2 / ell_s^3 exp(...) v_j
    (Sec. 3.3, eq. "add_gauss_kernel" and the derivative formula after it)."""
    X = np.ascontiguousarray(points, dtype=np.float32)
    N, d = X.shape
    P = len(windows)
    rows = np.arange(N, dtype=np.int64) if rows is None else np.ascontiguousarray(rows, dtype=np.int64)
    off, feat = _csr(windows)
    ell = np.ascontiguousarray(ell, dtype=np.float64)
    v = np.ascontiguousarray(v, dtype=np.float64)
    Kv = np.zeros(len(rows))
    dK = np.zeros((P, len(rows)))
    L = _clib.lib()
    L.orc_direct(N, d, _clib.ptr(X), P, _clib.ptr(off), _clib.ptr(feat), _clib.ptr(ell), float(sigma_f),
                 _clib.ptr(v), len(rows), _clib.ptr(rows), _clib.ptr(Kv), _clib.ptr(dK))
    return Kv, dK


def adjoint_exact(x: np.ndarray, v: np.ndarray, M: int) -> np.ndarray:
    """S_k = sum_j v_j exp(-2 pi i k.x_j) for k in I_M^d, exactly (array indexed k + M/2)."""
    x = np.asarray(x, dtype=np.float64)
    d = x.shape[1]
    k = np.arange(-M // 2, M // 2)
    E = [np.exp(-2j * np.pi * np.outer(x[:, t], k)) for t in range(d)]
    if d == 1:
        return v @ E[0]
    if d == 2:
        return np.einsum("j,ja,jb->ab", v, E[0], E[1], optimize=True)
    out = np.zeros((M, M, M), dtype=np.complex128)
    for s in range(0, x.shape[0], 512):
        e = slice(s, s + 512)
        A = (v[e, None] * E[0][e])                              # j x a
        B = (E[1][e, :, None] * E[2][e, None, :]).reshape(-1, M * M)   # j x (b c)
        out += (A.T @ B).reshape(M, M, M)
    return out


def forward_exact(x: np.ndarray, dhat: np.ndarray) -> np.ndarray:
    """f(x_i) = sum_{k in I_M^d} dhat_k exp(+2 pi i k.x_i), exactly (complex)."""
    x = np.asarray(x, dtype=np.float64)
    d = x.shape[1]
    M = dhat.shape[0]
    k = np.arange(-M // 2, M // 2)
    E = [np.exp(2j * np.pi * np.outer(x[:, t], k)) for t in range(d)]
    if d == 1:
        return E[0] @ dhat
    if d == 2:
        return np.einsum("na,ab,nb->n", E[0], dhat, E[1], optimize=True)
    tmp = (dhat.reshape(M * M, M) @ E[2].T).reshape(M, M, -1)
    tmp = np.einsum("abn,nb->an", tmp, E[1])
    return np.einsum("an,na->n", tmp, E[0])


def ndft_fastsum(x: np.ndarray, v: np.ndarray, chats) -> list:
    """Level 2: h~(x_i) = sum_k c_hat_k S_k exp(2 pi i k.x_i) for each c_hat in chats."""
    S = adjoint_exact(x, np.asarray(v, dtype=np.float64), chats[0].shape[0])
    return [forward_exact(x, c * S).real for c in chats]


@functools.lru_cache(maxsize=64)
def _phihat_grid(M: int, n: int, m: int, sigma: float, d: int, win: str = "kb") -> np.ndarray:
    """prod_t phi_hat(k_t) on I_M^d (the window transform depends only on the settings: computed once
    per setting and kept, like the setup of a plan; callers do not modify it)."""
    ph = window.phihat_quadrature(np.arange(-M // 2, M // 2), n, m, sigma, window=win)
    out = ph
    for _ in range(d - 1):
        out = np.multiply.outer(out, ph)
    return out


def nfft_adjoint(x: np.ndarray, v: np.ndarray, M: int, n: int, m: int, sigma: float = 2.0, win: str = "kb"):
    """Approximate S_k, k in I_M^d: spread, n^d FFT, keep I_M, divide by n^d prod phi_hat."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    N, d = x.shape
    v = np.ascontiguousarray(v, dtype=np.float64)
    g = np.zeros((n,) * d)
    _clib.lib().orc_spread(N, d, _clib.ptr(x), _clib.ptr(v), n, m, window.shape_of(m, sigma, win),
                           window.KINDS[win], _clib.ptr(g))
    G = np.fft.fftshift(np.fft.fftn(np.fft.ifftshift(g)))          # index k + n/2, k in I_n
    sl = tuple([slice(n // 2 - M // 2, n // 2 + M // 2)] * d)
    return G[sl] / (n ** d * _phihat_grid(M, n, m, sigma, d, win))


def nfft_forward(x: np.ndarray, dhats, n: int, m: int, sigma: float = 2.0, win: str = "kb") -> np.ndarray:
    """Approximate f_q(x_i) = sum_k dhat_q,k exp(2 pi i k.x_i) for each dhat_q (real part kept):
    divide by n^d prod phi_hat, zero-pad to I_n, inverse n^d FFT, interpolate."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    N, d = x.shape
    M = dhats[0].shape[0]
    sl = tuple([slice(n // 2 - M // 2, n // 2 + M // 2)] * d)
    phg = _phihat_grid(M, n, m, sigma, d, win)
    hs = []
    for dh in dhats:
        ghat = np.zeros((n,) * d, dtype=np.complex128)
        ghat[sl] = dh / (n ** d * phg)
        h = np.fft.fftshift(np.fft.ifftn(np.fft.ifftshift(ghat))) * n ** d    # h_l, l in I_n
        hs.append(h.real)
    H = np.ascontiguousarray(np.stack(hs))
    out = np.zeros((len(dhats), N))
    _clib.lib().orc_gather(N, d, _clib.ptr(x), n, m, window.shape_of(m, sigma, win), window.KINDS[win],
                           len(dhats), _clib.ptr(H), _clib.ptr(out))
    return out


def nfft_fastsum(x: np.ndarray, v: np.ndarray, chats, n: int, m: int, sigma: float = 2.0,
                 targets: np.ndarray | None = None, win: str = "kb") -> np.ndarray:
    """Level 3: adjoint NFFT -> multiply by c_hat -> NFFT, for each c_hat in chats (rows of the result).
    The sums are evaluated at `targets` (the x'_i of eq. "fast sum"), by default at the sources x."""
    M = chats[0].shape[0]
    S = nfft_adjoint(x, v, M, n, m, sigma, win)
    return nfft_forward(x if targets is None else targets, [c * S for c in chats], n, m, sigma, win)


KINDS = {"gauss": ("gauss", "der", 2.0), "matern": ("matern", "matern_der", 1.0)}


def window_coefficients(ell: float, d: int, M: int, p: int, eps_B: float, kernel: str = "gauss"):
    """Coefficients of the kernel and its derivative kernel under the radial reading (degree p)."""
    kk, kd, _ = KINDS[kernel]
    return (kernels.coefficients(ell, d, M, p, eps_B, kk),
            kernels.coefficients(ell, d, M, p, eps_B, kd))


def default_reg(kernel: str) -> str:
    """The separable reading for the Gaussian family, the radial one for Matern(1/2) (not separable)."""
    return "separable" if kernel == "gauss" else "radial"


def coefficients_for(xs: np.ndarray, ell: float, M: int, p=None, eps_B: float = 1.0 / 16.0,
                     kernel: str = "gauss", reg: str | None = None, split: bool = True):
    """(c_hat, c_hat^der, q) of one window whose source points (N x d_s, the window's coordinates) are xs.

    reg 'separable' (default for the Gaussian): kernels.coefficients_separable on the fit intervals
    a_t of every axis, computed from the largest |coordinate| of xs; reg 'radial': the radial
    regularisation of degree p (kernels.default_p when None). Under the separable reading the window's
    quadratic part is split off when kernels.split_quadratic says so (and `split` allows it): then
    c_hat^der is the remainder's, and q = 1/(2 ell^2) is the weight of kernels.quadratic_part that every
    derivative product adds; q = 0 otherwise."""
    reg = default_reg(kernel) if reg is None else reg
    d = xs.shape[1]
    if reg == "separable":
        if kernel != "gauss":
            raise ValueError("the separable reading covers the Gaussian family only")
        maxabs = np.abs(xs).max(axis=0) if xs.shape[0] else np.zeros(d)
        iv = [kernels.fit_interval(float(a), M, eps_B) for a in maxabs]
        cg = kernels.coefficients_separable(ell, M, iv, "gauss")
        cd = kernels.coefficients_separable(ell, M, iv, "der")
        cp = kernels.coefficients_separable(ell, M, iv, "quad")
        if split and kernels.split_quadratic(cd, cp):
            return cg, cd - cp, 1.0 / (2.0 * ell * ell)
        return cg, cd, 0.0
    if reg != "radial":
        raise ValueError(reg)
    ps = kernels.default_p(M, eps_B) if p is None else int(p)
    return window_coefficients(ell, d, M, ps, eps_B, kernel) + (0.0,)


def direct_matern(points, windows, ell, sigma_f: float, v, rows=None, block: int = 256):
    """Direct FP64 sums of the additive Matern(1/2) kernel (Sec. 5): (K v)_i = sigma_f^2 sum_s sum_j
    exp(-r_s/ell_s) v_j and (dK/d ell_s v)_i = sigma_f^2 sum_j (r_s/ell_s^2) exp(-r_s/ell_s) v_j,
    r_s = ||x_i^W_s - x_j^W_s||; numpy, row blocks."""
    X = np.asarray(points, dtype=np.float32).astype(np.float64)
    v = np.asarray(v, dtype=np.float64)
    rows = np.arange(X.shape[0]) if rows is None else np.asarray(rows)
    P = len(windows)
    Kv = np.zeros(len(rows))
    dK = np.zeros((P, len(rows)))
    for b0 in range(0, len(rows), block):
        rb = rows[b0:b0 + block]
        for s, w in enumerate(windows):
            Y = X[:, list(w)]
            r = np.sqrt(np.sum((Y[rb][:, None, :] - Y[None, :, :]) ** 2, axis=2))
            E = np.exp(-r / ell[s])
            Kv[b0:b0 + block] += sigma_f ** 2 * (E @ v)
            dK[s, b0:b0 + block] = sigma_f ** 2 * ((r / ell[s] ** 2 * E) @ v)
    return Kv, dK


def matvec_all(points, windows, ell, sigma_f: float, v, bandwidth, cutoff: int, p=None,
               eps_B: float = 1.0 / 16.0, sigma: float = 2.0, level: str = "nfft", rows=None,
               kernel: str = "gauss", win: str = "kb", reg: str | None = None, coefs=None, split: bool = True):
    """Fused product: returns (K v, dK/d ell [P, .]) at level 'nfft' (CPU NFFT fast sum)
    or 'ndft' (exact trigonometric sum). v is one right-hand side of length N. With `rows`, the
    outputs are evaluated only at those points (all N points are still sources). `win` selects the
    NFFT window ('kb' Kaiser-Bessel, 'es' exponential of semicircle); `reg` the reading of the
    regularisation (coefficients_for), `split` whether a window's quadratic part may be split off.
    `coefs` may hold the P triples (c_hat, c_hat^der, q) from an earlier call (they depend only on the
    points' extents and the hyperparameters)."""
    X = np.asarray(points, dtype=np.float32).astype(np.float64)
    v = np.asarray(v, dtype=np.float64)
    P = len(windows)
    if np.isscalar(bandwidth):
        bandwidth = [int(bandwidth)] * P
    T = X if rows is None else X[np.asarray(rows)]
    N = T.shape[0]
    Kv = np.zeros(N)
    dK = np.zeros((P, N))
    for s, w in enumerate(windows):
        d = len(w)
        M = int(bandwidth[s])
        xs = np.ascontiguousarray(X[:, list(w)])
        if coefs is not None:
            cg, cd, q = coefs[s]
        else:
            cg, cd, q = coefficients_for(xs, float(ell[s]), M, p, eps_B, kernel, reg, split)
        xt = None if rows is None else np.ascontiguousarray(T[:, list(w)])
        if level == "nfft":
            outK, outD = nfft_fastsum(xs, v, [cg, cd], int(round(sigma * M)), cutoff, sigma, targets=xt, win=win)
        elif level == "ndft":
            if rows is not None:
                raise ValueError("rows are supported at level 'nfft' only")
            outK, outD = ndft_fastsum(xs, v, [cg, cd])
        else:
            raise ValueError(level)
        if q:
            outD = outD + q * kernels.quadratic_part(xs, v, None if rows is None else xt)
        Kv += sigma_f ** 2 * outK
        dK[s] = sigma_f ** 2 * (KINDS[kernel][2] / ell[s]) * outD
    return Kv, dK
