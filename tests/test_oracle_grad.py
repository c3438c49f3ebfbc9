"""Pins for the oracle's gradients of f = w^T K(theta) v: finite differences of the direct FP64
objective and of the oracle's own NFFT objective, and their agreement at the method's error level."""
import numpy as np
import pytest

import workloads
from oracle import fastsum, gradients


@pytest.fixture(scope="module")
def case():
    wl = workloads.tiny(N=60, d=5, windows=[(0, 1, 2), (3, 4)], ell=[0.3, 0.2])
    v = wl.vector().astype(np.float64)
    w = wl.vector(which=2).astype(np.float64)
    return wl, v, w


def f_direct(X, wl, v, w, ell=None, sigma_f=None):
    Kv, _ = fastsum.direct(X, wl.windows, wl.ell if ell is None else ell, wl.sigma_f if sigma_f is None else sigma_f, v)
    return w @ Kv


def test_direct_point_gradient_is_finite_difference(case):
    wl, v, w = case
    _, _, _, gx = gradients.direct_grad(wl.points, wl.windows, wl.ell, wl.sigma_f, v, w)
    X = wl.points.astype(np.float64)
    h = 1e-6
    for k, f in [(0, 0), (7, 2), (33, 3), (59, 4), (20, 1)]:
        Xp, Xm = X.copy(), X.copy()
        Xp[k, f] += h
        Xm[k, f] -= h
        # the direct sum takes float32 points: difference in FP64 by evaluating with float64 arrays
        fd = (f_direct64(Xp, wl, v, w) - f_direct64(Xm, wl, v, w)) / (2 * h)
        assert gx[k, f] == pytest.approx(fd, rel=1e-6, abs=1e-8)


def f_direct64(X, wl, v, w):
    """w^T K v with float64 points (a plain numpy evaluation of the definition)."""
    tot = 0.0
    for s, win in enumerate(wl.windows):
        Y = X[:, list(win)]
        D2 = ((Y[:, None, :] - Y[None, :, :]) ** 2).sum(-1)
        tot += w @ (np.exp(-D2 / (2 * wl.ell[s] ** 2)) @ v)
    return wl.sigma_f ** 2 * tot


def test_direct_parameter_gradients(case):
    wl, v, w = case
    gv, gell, gsf, _ = gradients.direct_grad(wl.points, wl.windows, wl.ell, wl.sigma_f, v, w)
    Kw, _ = fastsum.direct(wl.points, wl.windows, wl.ell, wl.sigma_f, w)
    np.testing.assert_allclose(gv, Kw)
    for s in range(wl.P):
        ep, em = wl.ell.copy(), wl.ell.copy()
        ep[s] += 1e-6
        em[s] -= 1e-6
        fd = (f_direct(wl.points, wl, v, w, ell=ep) - f_direct(wl.points, wl, v, w, ell=em)) / 2e-6
        assert gell[s] == pytest.approx(fd, rel=1e-6)
    fd = (f_direct(wl.points, wl, v, w, sigma_f=wl.sigma_f + 1e-6) - f_direct(wl.points, wl, v, w, sigma_f=wl.sigma_f - 1e-6)) / 2e-6
    assert gsf == pytest.approx(fd, rel=1e-6)


def f_nfft(X, wl, v, w, M, m):
    Kv, _ = fastsum.matvec_all(X, wl.windows, wl.ell, wl.sigma_f, v, M, m)
    return w @ Kv


def test_nfft_point_gradient_is_finite_difference_of_nfft_objective():
    """The NFFT gradient is the exact derivative of the approximate objective: moving x_k moves both
    its spreading and its interpolation, and the two window-derivative gathers account for both."""
    wl = workloads.tiny(N=80, d=3, windows=[(0, 1, 2)], ell=[0.35])
    v = wl.vector().astype(np.float64)
    w = wl.vector(which=2).astype(np.float64)
    M, m = 16, 4
    _, _, _, gx = gradients.nfft_grad(wl.points, wl.windows, wl.ell, wl.sigma_f, v, w, M, m)
    X = wl.points.astype(np.float64)
    h = 2.0 ** -17          # the product takes float32 points; x +- h is exact in float32 for |x| < 1/4
    for k, f in [(0, 0), (13, 1), (79, 2), (40, 0)]:
        Xp, Xm = X.copy(), X.copy()
        Xp[k, f] += h
        Xm[k, f] -= h
        fd = (f_nfft(Xp, wl, v, w, M, m) - f_nfft(Xm, wl, v, w, M, m)) / (2 * h)
        assert gx[k, f] == pytest.approx(fd, rel=2e-5, abs=1e-7)


def test_gather_gradient_is_finite_difference():
    rng = np.random.default_rng(2)
    n, m = 32, 4
    h = rng.standard_normal((n, n))
    x = rng.uniform(-0.2, 0.2, (20, 2))
    val, grad = gradients.gather_grad(x, h, n, m)
    eps = 1e-7
    for t in range(2):
        xp, xm = x.copy(), x.copy()
        xp[:, t] += eps
        xm[:, t] -= eps
        fd = (gradients.gather_grad(xp, h, n, m)[0] - gradients.gather_grad(xm, h, n, m)[0]) / (2 * eps)
        np.testing.assert_allclose(grad[:, t], fd, rtol=1e-5, atol=1e-6 * np.abs(grad).max())


def test_nfft_gradients_approach_direct_ones():
    wl = workloads.make("c0", N=400)
    v = wl.vector().astype(np.float64)
    w = wl.vector(which=2).astype(np.float64)
    a = gradients.nfft_grad(wl.points, wl.windows, wl.ell, wl.sigma_f, v, w, 32, 4)
    b = gradients.direct_grad(wl.points, wl.windows, wl.ell, wl.sigma_f, v, w)
    rel = lambda x, y: np.linalg.norm(np.ravel(x) - np.ravel(y)) / np.linalg.norm(np.ravel(y))
    assert rel(a[0], b[0]) < 3e-3 and rel(a[1], b[1]) < 1e-2 and rel(a[2], b[2]) < 3e-3
    assert rel(a[3], b[3]) < 5e-2
