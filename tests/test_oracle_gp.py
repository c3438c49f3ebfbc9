"""Pins of oracle/gp.py (CG, log marginal likelihood and its gradient, Hutchinson estimator) against
things other than themselves: numpy's dense solver, central finite differences of the log marginal
likelihood, the exact trace (identity probes), and the estimator's expectation."""
import numpy as np
import pytest

import workloads
from oracle import fastsum, gp


def small(N=120, seed=5):
    wl = workloads.tiny(N=N, d=5, windows=[(0, 1, 2), (3, 4)], seed=seed, ell=[0.3, 0.45])
    return wl


def test_cg_matches_dense_solve():
    wl = small()
    K, _ = gp.dense_kernel(wl.points, wl.windows, wl.ell, wl.sigma_f)
    A = K + 0.7 * np.eye(wl.N)
    Y = np.random.default_rng(1).standard_normal((wl.N, 3))
    X, iters, rel = gp.cg(lambda V: A @ V, Y, 1e-12, 1000)
    assert np.all(rel <= 1e-12) and np.all(iters > 0)
    assert np.linalg.norm(X - np.linalg.solve(A, Y)) <= 1e-9 * np.linalg.norm(X)
    # single column and an already-solved column (y = 0 stops at once)
    x1, it1, r1 = gp.cg(lambda V: A @ V, Y[:, 0], 1e-12, 1000)
    assert np.allclose(x1, X[:, 0]) and it1 == iters[0]


def test_cg_stops_at_tolerance():
    wl = small()
    K, _ = gp.dense_kernel(wl.points, wl.windows, wl.ell, wl.sigma_f)
    A = K + 0.05 * np.eye(wl.N)
    y = np.random.default_rng(2).standard_normal(wl.N)
    x, it, rel = gp.cg(lambda V: A @ V, y, 1e-3, 1000)
    assert rel <= 1e-3 and np.linalg.norm(y - A @ x) <= 1e-3 * np.linalg.norm(y) * (1 + 1e-9)
    x2, it2, _ = gp.cg(lambda V: A @ V, y, 1e-3, it - 1)           # one iteration short: not converged
    assert np.linalg.norm(y - A @ x2) > 1e-3 * np.linalg.norm(y)


def test_dense_kernel_matches_direct_sums():
    from oracle import fastsum
    wl = small()
    K, dK = gp.dense_kernel(wl.points, wl.windows, wl.ell, wl.sigma_f)
    v = np.random.default_rng(3).standard_normal(wl.N)
    Kv, dKv = fastsum.direct(wl.points, wl.windows, wl.ell, wl.sigma_f, v)
    assert np.allclose(K @ v, Kv, rtol=1e-12, atol=1e-12)
    assert np.allclose(np.einsum("sij,j->si", dK, v), dKv, rtol=1e-12, atol=1e-12)


def test_lml_gradient_matches_finite_differences():
    """Central differences of L in each of ell_s, sigma_f, beta (h = 1e-5; FP64, agreement ~1e-7)."""
    wl = small()
    y = np.random.default_rng(4).standard_normal(wl.N)
    beta = 0.3

    def L(ell, sf, b):
        K, _ = gp.dense_kernel(wl.points, wl.windows, ell, sf)
        return gp.lml(K, b, y)

    K, dK = gp.dense_kernel(wl.points, wl.windows, wl.ell, wl.sigma_f)
    g = gp.lml_grad_exact(K, dK, wl.sigma_f, beta, y)
    h = 1e-5
    fd = []
    for s in range(wl.P):
        ep, em = wl.ell.copy(), wl.ell.copy()
        ep[s] += h
        em[s] -= h
        fd.append((L(ep, wl.sigma_f, beta) - L(em, wl.sigma_f, beta)) / (2 * h))
    fd.append((L(wl.ell, wl.sigma_f + h, beta) - L(wl.ell, wl.sigma_f - h, beta)) / (2 * h))
    fd.append((L(wl.ell, wl.sigma_f, beta + h) - L(wl.ell, wl.sigma_f, beta - h)) / (2 * h))
    assert np.allclose(g, fd, rtol=1e-6, atol=1e-6 * np.abs(fd).max())


def test_lml_matches_slogdet_definition():
    wl = small()
    K, _ = gp.dense_kernel(wl.points, wl.windows, wl.ell, wl.sigma_f)
    y = np.random.default_rng(6).standard_normal(wl.N)
    A = K + 0.4 * np.eye(wl.N)
    ref = -0.5 * y @ np.linalg.solve(A, y) - 0.5 * np.linalg.slogdet(A)[1] - 0.5 * wl.N * np.log(2 * np.pi)
    assert abs(gp.lml(K, 0.4, y) - ref) <= 1e-10 * abs(ref)


def test_hutchinson_with_identity_probes_is_exact():
    """Z = I (m = N probes): the estimator equals the exact trace."""
    wl = small(N=60)
    K, dK = gp.dense_kernel(wl.points, wl.windows, wl.ell, wl.sigma_f)
    y = np.random.default_rng(7).standard_normal(wl.N)
    g = gp.lml_grad_exact(K, dK, wl.sigma_f, 0.2, y)
    # 1/m with m = N scales the estimator; identity probes times sqrt(N) make (1/m) sum z z^T = I
    h = gp.lml_grad_hutchinson_dense(K, dK, wl.sigma_f, 0.2, y, np.sqrt(wl.N) * np.eye(wl.N))
    assert np.allclose(h, g, rtol=1e-10, atol=1e-10 * np.abs(g).max())


def test_hutchinson_is_unbiased():
    """Averaged over many Rademacher probes the estimate approaches the exact gradient (the trace
    term's standard error shrinks like 1/sqrt(m))."""
    wl = small(N=80)
    K, dK = gp.dense_kernel(wl.points, wl.windows, wl.ell, wl.sigma_f)
    y = np.random.default_rng(8).standard_normal(wl.N)
    g = gp.lml_grad_exact(K, dK, wl.sigma_f, 0.5, y)
    Z = np.random.default_rng(9).choice([-1.0, 1.0], size=(wl.N, 20000))
    h = gp.lml_grad_hutchinson_dense(K, dK, wl.sigma_f, 0.5, y, Z)
    assert np.allclose(h, g, rtol=0.02, atol=0.02 * np.abs(g).max())


def test_product_form_equals_dense_form():
    """lml_grad_hutchinson (CG + products) equals the dense estimator for the same probes."""
    wl = small()
    K, dK = gp.dense_kernel(wl.points, wl.windows, wl.ell, wl.sigma_f)
    y = np.random.default_rng(10).standard_normal(wl.N)
    Z = np.random.default_rng(11).choice([-1.0, 1.0], size=(wl.N, 4))

    def apply_all(V):
        return K @ V, [dK[s] @ V for s in range(wl.P)]

    g, alpha, _ = gp.lml_grad_hutchinson(apply_all, wl.sigma_f, 0.6, y, Z, 1e-13, 2000)
    h = gp.lml_grad_hutchinson_dense(K, dK, wl.sigma_f, 0.6, y, Z)
    assert np.allclose(g, h, rtol=1e-8, atol=1e-8 * np.abs(h).max())
    assert np.allclose(alpha, np.linalg.solve(K + 0.6 * np.eye(wl.N), y), rtol=1e-9, atol=1e-9)


def test_planted_gradient_mistakes_are_caught(monkeypatch):
    """The finite-difference pin has teeth: a dropped 2/sigma_f factor or a flipped trace sign fails it."""
    wl = small()
    y = np.random.default_rng(12).standard_normal(wl.N)
    K, dK = gp.dense_kernel(wl.points, wl.windows, wl.ell, wl.sigma_f)
    h = 1e-5
    fd_sf = (gp.lml(gp.dense_kernel(wl.points, wl.windows, wl.ell, wl.sigma_f + h)[0], 0.3, y) -
             gp.lml(gp.dense_kernel(wl.points, wl.windows, wl.ell, wl.sigma_f - h)[0], 0.3, y)) / (2 * h)
    good = gp.lml_grad_exact(K, dK, wl.sigma_f, 0.3, y)
    assert abs(good[wl.P] - fd_sf) <= 1e-6 * abs(fd_sf)
    real = gp._derivatives
    monkeypatch.setattr(gp, "_derivatives", lambda K, dK, sf: real(K, dK, sf)[:-2] + [K, np.eye(K.shape[0])])
    assert abs(gp.lml_grad_exact(K, dK, wl.sigma_f, 0.3, y)[wl.P] - fd_sf) > 1e-3 * abs(fd_sf)
    monkeypatch.setattr(gp, "_derivatives", real)
    g_flip = np.array([0.5 * a + 0.5 * b for a, b in zip(
        [np.linalg.solve(K + 0.3 * np.eye(wl.N), y) @ D @ np.linalg.solve(K + 0.3 * np.eye(wl.N), y)
         for D in real(K, dK, wl.sigma_f)],
        [np.trace(np.linalg.solve(K + 0.3 * np.eye(wl.N), D)) for D in real(K, dK, wl.sigma_f)])])
    assert not np.allclose(g_flip, good, rtol=1e-3)


# ---------------------------------------------------------------- preconditioned CG ----

def test_woodbury_apply_is_the_dense_inverse():
    rng = np.random.default_rng(21)
    U = rng.standard_normal((80, 7))
    w = rng.uniform(0.5, 3.0, 7)
    beta = 0.03
    r = rng.standard_normal((80, 2))
    B = beta * np.eye(80) + U @ np.diag(w) @ U.T
    np.testing.assert_allclose(gp.woodbury_apply(U, w, beta)(r), np.linalg.solve(B, r), rtol=1e-9, atol=1e-9)


def test_fourier_basis_is_the_trig_sum_of_the_retained_modes():
    """U diag(w) U^T equals sigma_f^2 sum over the retained (window, +-k) of c_hat_k e^{2 pi i k.(x_i - x_j)},
    the constant mode counted once per window (cos(a - b) = cos a cos b + sin a sin b)."""
    wl = workloads.tiny(N=40, d=5, windows=[(0, 1, 2), (3, 4)], ell=[0.3, 0.6])
    X = wl.points.astype(np.float64)
    coefs = [fastsum.coefficients_for(np.ascontiguousarray(X[:, list(w)]), wl.ell[s], 16)[0]
             for s, w in enumerate(wl.windows)]
    beta, sf = 1e-3, 1.3
    modes, wmode = gp.fourier_modes(wl.windows, coefs, 1, beta, sf, 40)
    U, owner = gp.fourier_basis(wl.points, wl.windows, modes)
    got = U @ np.diag(wmode[owner]) @ U.T
    want = np.zeros((40, 40))
    for s, w in enumerate(wl.windows):
        c = coefs[s]
        M = c.shape[0]
        xs = X[:, list(w)]
        for k in np.ndindex(*c.shape):
            kk = np.array(k) - M // 2
            keep = np.all(kk == 0) or (s, tuple(kk)) in modes or (s, tuple(-kk)) in modes
            if keep:
                ph = 2 * np.pi * (xs @ kk)
                want += sf ** 2 * c[k] * np.cos(ph[:, None] - ph[None, :])
    np.testing.assert_allclose(got, want, rtol=1e-10, atol=1e-10)
    assert len(modes) > 1 and all(wm > 0 for wm in wmode)


def test_pcg_with_identity_is_cg():
    rng = np.random.default_rng(22)
    Q = rng.standard_normal((60, 60))
    A = Q @ Q.T + 0.5 * np.eye(60)
    y = rng.standard_normal(60)
    x1, it1, r1 = gp.cg(lambda v: A @ v, y, 1e-10, 500)
    x2, it2, r2 = gp.pcg(lambda v: A @ v, lambda v: v, y, 1e-10, 500)
    # with M = I the flexible and the classical direction updates agree in exact arithmetic; in FP64 the
    # iteration counts may differ by one
    assert abs(it1 - it2) <= 2 and r2 <= 1e-10
    np.testing.assert_allclose(x1, x2, rtol=1e-8, atol=1e-10)


def test_fourier_preconditioner_on_the_gp_configuration():
    """The GP configuration's points (a 1500-point sample, 8 windows of 3, ell = 0.5) at the configuration's
    noise variance beta = 0.01: preconditioned CG reaches the dense solution in a fraction of plain CG's
    iterations."""
    wl = workloads.make("c4", N=2_000_000)
    idx = np.random.default_rng(23).choice(wl.N, 1500, replace=False)
    X = wl.points[idx]
    y = wl.targets()[idx].astype(np.float64)
    K, _ = gp.dense_kernel(X, wl.windows, wl.ell, wl.sigma_f)
    beta = 0.01
    A = K + beta * np.eye(len(y))
    x_ref = np.linalg.solve(A, y)
    coefs = [fastsum.coefficients_for(np.ascontiguousarray(wl.points[:, list(w)].astype(np.float64)), wl.ell[s], 32)[0]
             for s, w in enumerate(wl.windows)]
    modes, wmode = gp.fourier_modes(wl.windows, coefs, 1, beta, wl.sigma_f, len(y))
    U, owner = gp.fourier_basis(X, wl.windows, modes)
    Minv = gp.woodbury_apply(U, wmode[owner], beta)
    xp, itp, rp = gp.pcg(lambda v: A @ v, Minv, y, 1e-8, 500)
    xc, itc, rc = gp.cg(lambda v: A @ v, y, 1e-8, 2000)
    assert rp <= 1e-8 and np.linalg.norm(xp - x_ref) <= 1e-5 * np.linalg.norm(x_ref)
    assert itp * 3 < itc
