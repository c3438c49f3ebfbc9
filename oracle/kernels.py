"""Gaussian and derivative-Gaussian kernels, their regularisation and their
discrete Fourier coefficients, FP64. Test infrastructure only.

Kernels (Sec. 3.3, eqs. "implement_gaussian_kernel" and
"implement_der_gaussian_kernel", with c = sqrt(2) ell):

    kappa_gauss(r) = exp(-r^2 / c^2)
    kappa_der(r)   = (r^2 / c^2) exp(-r^2 / c^2)

so that K v = sigma_f^2 sum_s K_s^gauss v and dK/d ell_s v = sigma_f^2 (2/ell_s) K_s^der v.

Matern(1/2) (Sec. 5, "Extension to Other Kernels"): kappa_M(r) = exp(-r/ell) and the derivative
kernel kappa_derM(r) = (r/ell) exp(-r/ell), so that dK/d ell_s v = sigma_f^2 (1/ell_s) K_s^derM v
(kinds 'matern' and 'matern_der'). The same boundary regularisation is applied; the kink of
exp(-r/ell) at r = 0 stays (no near-field correction, which the paper does not describe), so its
coefficients decay slowly and the Fourier approximation is far less accurate than the Gaussian's.

Regularisation (Sec. 3.1: a smoother periodisation, the kernel smoothed near the
boundary of the period, after Potts-Steidl; the paper does not write it down). Reading: with
a = 1/2 - eps_B the regularised radial profile is

    K_R(r) = kappa(r)           r <= a
           = T(r)               a < r <= 1/2
           = kappa(1/2)         r > 1/2 (inside the cube [-1/2,1/2]^d)

where T is the polynomial of degree 2p-1 with T^(j)(a) = kappa^(j)(a) for
j < p, T(1/2) = kappa(1/2) and T^(j)(1/2) = 0 for 1 <= j < p. p = 0 means no
regularisation at all: K_R = kappa on the whole cube, i.e. the plain periodic
continuation that the error theorems of Sec. 3.4 assume.

Discrete Fourier coefficients (Lemma "aliasing error", Sec. 3.4):

    c_hat_k = M^-d sum_{j in I_M} K_R(||j/M||) exp(-2 pi i j.k / M),   k in I_M,
    I_M = {-M/2, ..., M/2-1}^d.

Separable reading (the default for the Gaussian family). Sec. 3.4 ("Gaussian Kernel") writes the
Gaussian's coefficients as the tensor product c_k = c_k1(f) c_k2(f) c_k3(f), f(x) = exp(-x^2/(2 ell^2)),
and ("Derivative Gaussian Kernel") the derivative kernel's as the three-term sum
c_k1(g) c_k2(f) c_k3(f) + c_k1(f) c_k2(g) c_k3(f) + c_k1(f) c_k2(f) c_k3(g), g(x) = x^2/(2 ell^2) f(x).
Here each 1-D factor is replaced by its Fourier extension (Boyd 2002, "A comparison of numerical
algorithms for Fourier extension of the first, second, and third kinds"; Huybrechs 2010, "On the
Fourier extension of nonperiodic functions"): the even trigonometric polynomial of degree < M/2 that
fits f (or g) in the least-squares sense on the interval [0, a_t] that holds every coordinate
difference of axis t, and is free outside it. This is the paper's "regularised at the edges by a smooth
transition" taken per axis, with the transition chosen by the fit instead of prescribed:

    a_t = min(1/2 - eps_B, max(a_lo(M), 2 max_j |x_{j,t}|)),   a_lo(M) = max(1/4, 1/2 - 4/M),

since |x_{i,t} - x_{j,t}| <= 2 max_j |x_{j,t}| <= 1/2 - eps_B for points in the ball of radius
1/4 - eps_B/2. The floor a_lo keeps the least-squares problem well conditioned (condition number of
the cosine basis below ~1e5); on [0, a_lo] the fit error is already below 1e-8.
"""
from __future__ import annotations

from math import factorial

import numpy as np
from numpy.polynomial.hermite import hermval


def kappa(r, ell: float, kind: str = "gauss"):
    """kind='gauss': exp(-r^2/c^2); kind='der': (r^2/c^2) exp(-r^2/c^2); c = sqrt(2) ell;
    kind='matern': exp(-r/ell); kind='matern_der': (r/ell) exp(-r/ell)."""
    r = np.asarray(r, dtype=np.float64)
    if kind in ("matern", "matern_der"):
        t = r / ell
        return np.exp(-t) if kind == "matern" else t * np.exp(-t)
    q = r * r / (2.0 * ell * ell)
    e = np.exp(-q)
    return e if kind == "gauss" else q * e


def radial_derivatives(r0: float, ell: float, p: int, kind: str = "gauss"):
    """d^j/dr^j kappa(r) at r0 for j = 0..p-1.

    Gaussian: d^j/dr^j exp(-(r/c)^2) = (-1/c)^j H_j(r/c) exp(-(r/c)^2), H_j the
    physicists' Hermite polynomials. Derivative kernel: Leibniz rule on
    (r/c)^2 * exp(-(r/c)^2). Matern: d^j/dr^j exp(-r/ell) = (-1/ell)^j exp(-r/ell) and, by the same
    rule, d^j/dr^j (r/ell) exp(-r/ell) = (-1/ell)^j exp(-r/ell) (r/ell - j)."""
    if kind in ("matern", "matern_der"):
        j = np.arange(p, dtype=np.float64)
        g = (-1.0 / ell) ** j * np.exp(-r0 / ell)
        return g if kind == "matern" else g * (r0 / ell - j)
    c = np.sqrt(2.0) * ell
    x = r0 / c
    g = []
    for j in range(p + 2):
        coef = np.zeros(j + 1)
        coef[j] = 1.0
        g.append((-1.0 / c) ** j * hermval(x, coef) * np.exp(-x * x))
    g = np.array(g)
    if kind == "gauss":
        return g[:p]
    q = [r0 * r0 / c ** 2, 2.0 * r0 / c ** 2, 2.0 / c ** 2]   # (r/c)^2 and its derivatives
    out = []
    for j in range(p):
        s = 0.0
        for i in range(0, min(j, 2) + 1):
            s += factorial(j) / (factorial(i) * factorial(j - i)) * q[i] * g[j - i]
        out.append(s)
    return np.array(out)


def transition_polynomial(ell: float, p: int, eps_B: float, kind: str = "gauss"):
    """Coefficients t_0..t_{2p-1} of T(r) = sum_i t_i (r - a)^i (see module docstring)."""
    a = 0.5 - eps_B
    h = 0.5 - a
    da = radial_derivatives(a, ell, p, kind)
    vb = float(kappa(0.5, ell, kind))
    n = 2 * p
    A = np.zeros((n, n))
    rhs = np.zeros(n)
    for j in range(p):                  # T^(j)(a) = kappa^(j)(a)
        A[j, j] = factorial(j)
        rhs[j] = da[j]
    for j in range(p):                  # T(1/2) = kappa(1/2), T^(j)(1/2) = 0 for j >= 1
        for i in range(j, n):
            A[p + j, i] = factorial(i) / factorial(i - j) * h ** (i - j)
        rhs[p + j] = vb if j == 0 else 0.0
    return np.linalg.solve(A, rhs)


def regularised(r, ell: float, p: int, eps_B: float, kind: str = "gauss"):
    """K_R(r) of the module docstring; p = 0 returns kappa itself."""
    r = np.asarray(r, dtype=np.float64)
    if p == 0:
        return kappa(r, ell, kind)
    a = 0.5 - eps_B
    t = transition_polynomial(ell, p, eps_B, kind)
    T = np.polynomial.polynomial.polyval(r - a, t)
    vb = float(kappa(0.5, ell, kind))
    return np.where(r <= a, kappa(r, ell, kind), np.where(r <= 0.5, T, vb))


def default_p(M: int, eps_B: float) -> int:
    """Regularisation degree used when none is given: about the number of coefficient-grid
    samples that fall in the transition band, M eps_B rounded half up, at least 1."""
    return max(1, int(np.floor(M * eps_B + 0.5)))


def coefficients(ell: float, d: int, M: int, p: int, eps_B: float, kind: str = "gauss"):
    """c_hat_k for k in I_M^d, as a real array of shape (M,)*d indexed by k + M/2.

    Samples K_R at j/M, j in I_M^d, then the d-dimensional DFT (Lemma "aliasing
    error"). The imaginary part vanishes because K_R is even; it is dropped."""
    j = np.arange(-M // 2, M // 2) / M
    grids = np.meshgrid(*([j] * d), indexing="ij")
    r = np.sqrt(sum(g * g for g in grids))
    samples = regularised(r, ell, p, eps_B, kind)
    c = np.fft.fftn(np.fft.ifftshift(samples)) / M ** d
    return np.fft.fftshift(c).real


def trig_poly_eval(chat: np.ndarray, r: np.ndarray) -> np.ndarray:
    """K_F(r) = sum_{k in I_M^d} c_hat_k exp(2 pi i k.r) at points r (npts x d)."""
    d = chat.ndim
    M = chat.shape[0]
    k = np.arange(-M // 2, M // 2)
    E = [np.exp(2j * np.pi * np.outer(r[:, t], k)) for t in range(d)]
    if d == 1:
        return (E[0] @ chat).real
    if d == 2:
        return np.einsum("na,ab,nb->n", E[0], chat, E[1]).real
    tmp = chat.reshape(M * M, M) @ E[2].T           # (a b) x n
    tmp = tmp.reshape(M, M, -1)
    tmp = np.einsum("abn,nb->an", tmp, E[1])
    return np.einsum("an,na->n", tmp, E[0]).real


# ------------------------------------------------------------------ separable reading ----

def fit_interval(maxabs: float, M: int, eps_B: float) -> float:
    """a_t of the module docstring for an axis whose largest |coordinate| is maxabs."""
    lo = max(0.25, 0.5 - 4.0 / M)
    return min(0.5 - eps_B, max(lo, 2.0 * float(maxabs)))


def extension_nodes(a: float, M: int) -> np.ndarray:
    """The J = 4M equispaced least-squares nodes a i/(J-1), i = 0..J-1, of [0, a]."""
    J = 4 * M
    return a * np.arange(J) / (J - 1)


def cosine_extension(values: np.ndarray, a: float, M: int) -> np.ndarray:
    """Least-squares Fourier extension of one even 1-D function from its values at extension_nodes(a, M):
    the b_k, k = 0..M/2-1, minimising sum_i (sum_k b_k cos(2 pi k x_i) - values_i)^2 (numpy's lstsq),
    returned as coefficients over I_M indexed k + M/2: c_0 = b_0, c_{+-k} = b_k/2, c_{-M/2} = 0."""
    x = extension_nodes(a, M)
    k = np.arange(M // 2)
    A = np.cos(2.0 * np.pi * np.outer(x, k))
    b, *_ = np.linalg.lstsq(A, np.asarray(values, dtype=np.float64), rcond=None)
    c = np.zeros(M)
    c[M // 2] = b[0]
    c[M // 2 + 1:] = b[1:] / 2.0
    c[1:M // 2] = b[:0:-1] / 2.0
    return c


def factor_coefficients(ell: float, a: float, M: int, kind: str = "gauss") -> np.ndarray:
    """1-D coefficients of f (kind 'gauss') or g (kind 'der') of the separable reading on [0, a]."""
    return cosine_extension(kappa(extension_nodes(a, M), ell, kind), a, M)


def coefficients_separable(ell: float, M: int, intervals, kind: str = "gauss") -> np.ndarray:
    """c_hat_k for k in I_M^d (d = len(intervals)), shape (M,)*d indexed k + M/2, of the separable
    reading: the tensor product of the 1-D factors (kind 'gauss') or the d-term sum with one factor g
    (kind 'der'), Sec. 3.4."""
    if kind not in ("gauss", "der", "quad"):
        raise ValueError("the separable reading covers the Gaussian family only")

    def outer(fs):
        out = fs[0]
        for q in fs[1:]:
            out = np.multiply.outer(out, q)
        return out

    d = len(intervals)
    if kind == "quad":
        # P(r) = ||r||^2 / (2 ell^2) = sum_t p(r_t): one factor p, the others the constant 1 (c_0 = 1)
        one = np.zeros(M)
        one[M // 2] = 1.0
        pf = [cosine_extension(extension_nodes(a, M) ** 2 / (2.0 * ell * ell), a, M) for a in intervals]
        return sum(outer([pf[t] if u == t else one for u in range(d)]) for t in range(d))
    f = [factor_coefficients(ell, a, M, "gauss") for a in intervals]
    if kind == "gauss":
        return outer(f)
    g = [factor_coefficients(ell, a, M, "der") for a in intervals]
    return sum(outer([g[t] if u == t else f[u] for u in range(d)]) for t in range(d))


# ------------------------------------------------------------ the quadratic part, split off ----
# For a wide kernel (ell large against the data) kappa_der(r) = q e^{-q}, q = ||r||^2/(2 ell^2), is close
# to its quadratic part P(r) = q. A trigonometric polynomial represents the quadratic on the torus with a
# large constant term that cancels against the low frequencies inside the data ball (about 24 times the
# product at ell = 1 on the benchmark's windows), which multiplies every FP32 rounding of the transforms
# by that factor. P is a rank-5 kernel, so P v needs no transform at all:
#     sum_j ||x_i - x_j||^2 v_j = ||x_i||^2 m0 - 2 x_i . m1 + m2,
#     m0 = sum_j v_j,  m1 = sum_j x_j v_j,  m2 = sum_j ||x_j||^2 v_j,
# and the fast summation then carries only the remainder R = kappa_der - P, whose coefficients are
# c_hat^der - c_hat^P (the same least-squares factors, kind 'quad'). For a narrow kernel R is no smaller
# than kappa_der and splitting would enlarge the transforms' terms instead, so a window is split only
# when that shrinks the constant coefficient: |c_0^der - c_0^P| < 0.9 |c_0^der|.

def split_quadratic(cd: np.ndarray, cp: np.ndarray) -> bool:
    """The rule above, from the coefficient arrays of kappa_der and of P (constant term at the centre)."""
    c = tuple(n // 2 for n in cd.shape)
    return abs(cd[c] - cp[c]) < 0.9 * abs(cd[c])


def quadratic_part(xs: np.ndarray, v: np.ndarray, targets: np.ndarray | None = None) -> np.ndarray:
    """sum_j ||x_i - x_j||^2 v_j for every target x_i (the sources xs by default), through the moments."""
    xs = np.asarray(xs, dtype=np.float64)
    v = np.asarray(v, dtype=np.float64)
    t = xs if targets is None else np.asarray(targets, dtype=np.float64)
    m0 = v.sum()
    m1 = xs.T @ v
    m2 = (xs * xs).sum(axis=1) @ v
    return (t * t).sum(axis=1) * m0 - 2.0 * (t @ m1) + m2
