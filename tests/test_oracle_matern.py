"""Pins of the Matern(1/2) kernels of the oracle (Sec. 5, "Extension to Other Kernels"):
closed forms, mpmath derivatives, the length-scale derivative identity kappa_der = ell d/d ell kappa,
brute-force direct sums, finite differences, and the convergence of the Fourier approximation."""
import mpmath
import numpy as np

import workloads
from oracle import fastsum, kernels


def test_kappa_closed_forms_and_ell_derivative():
    r = np.linspace(0.0, 0.7, 15)
    ell = 0.37
    assert np.allclose(kernels.kappa(r, ell, "matern"), np.exp(-r / ell), rtol=1e-15)
    h = 1e-6
    fd = (kernels.kappa(r, ell + h, "matern") - kernels.kappa(r, ell - h, "matern")) / (2 * h)
    # d/d ell exp(-r/ell) = (r/ell^2) exp(-r/ell) = kappa_der / ell
    assert np.allclose(ell * fd, kernels.kappa(r, ell, "matern_der"), rtol=1e-8, atol=1e-12)


def test_radial_derivatives_match_mpmath():
    ell, r0, p = 0.41, 0.4375, 6
    for kind, f in (("matern", lambda r: mpmath.exp(-r / ell)),
                    ("matern_der", lambda r: (r / ell) * mpmath.exp(-r / ell))):
        d = kernels.radial_derivatives(r0, ell, p, kind)
        ref = [float(mpmath.diff(f, mpmath.mpf(r0), j)) for j in range(p)]
        assert np.allclose(d, ref, rtol=1e-10, atol=1e-12), kind


def test_regularisation_conditions():
    ell, p, eps = 0.3, 3, 1.0 / 16
    a = 0.5 - eps
    for kind in ("matern", "matern_der"):
        t = kernels.transition_polynomial(ell, p, eps, kind)
        poly = np.polynomial.Polynomial(t)
        da = kernels.radial_derivatives(a, ell, p, kind)
        for j in range(p):
            assert abs(poly.deriv(j)(0.0) - da[j]) <= 1e-10 * max(1.0, abs(da[j]))
        assert abs(poly(eps) - kernels.kappa(0.5, ell, kind)) <= 1e-12
        for j in range(1, p):
            assert abs(poly.deriv(j)(eps)) <= 1e-8


def test_direct_sums_brute_force_and_fd():
    wl = workloads.tiny(N=25, d=4, windows=[(0, 1, 2), (3,)], seed=31, ell=[0.3, 0.2])
    v = wl.vector().astype(np.float64)
    Kv, dK = fastsum.direct_matern(wl.points, wl.windows, wl.ell, wl.sigma_f, v)
    X = wl.points.astype(np.float64)
    for i in (0, 7, 24):
        k = 0.0
        for s, w in enumerate(wl.windows):
            ds = 0.0
            for j in range(wl.N):
                r = np.sqrt(sum((X[i, f] - X[j, f]) ** 2 for f in w))
                k += wl.sigma_f ** 2 * np.exp(-r / wl.ell[s]) * v[j]
                ds += wl.sigma_f ** 2 * r / wl.ell[s] ** 2 * np.exp(-r / wl.ell[s]) * v[j]
            assert abs(dK[s, i] - ds) <= 1e-12 * max(1.0, abs(ds))
        assert abs(Kv[i] - k) <= 1e-12 * max(1.0, abs(k))
    h = 1e-6
    for s in range(wl.P):
        ep, em = wl.ell.copy(), wl.ell.copy()
        ep[s] += h
        em[s] -= h
        fd = (fastsum.direct_matern(wl.points, wl.windows, ep, wl.sigma_f, v)[0] -
              fastsum.direct_matern(wl.points, wl.windows, em, wl.sigma_f, v)[0]) / (2 * h)
        assert np.allclose(fd, dK[s], rtol=1e-6, atol=1e-8)
    w2 = wl.vector(which=2).astype(np.float64)
    Kw, _ = fastsum.direct_matern(wl.points, wl.windows, wl.ell, wl.sigma_f, w2)
    assert abs(w2 @ Kv - v @ Kw) <= 1e-12 * abs(v @ Kw)


def test_coefficient_derivative_identity():
    """c_hat of the regularised kappa_der equals ell d/d ell of c_hat of the regularised kappa (the
    regularisation is linear in the data and kappa_der = ell d/d ell kappa)."""
    ell, M, p, eps = 0.35, 16, 2, 1.0 / 16
    h = 1e-6
    fd = (kernels.coefficients(ell + h, 2, M, p, eps, "matern") -
          kernels.coefficients(ell - h, 2, M, p, eps, "matern")) / (2 * h)
    cd = kernels.coefficients(ell, 2, M, p, eps, "matern_der")
    assert np.allclose(ell * fd, cd, rtol=1e-6, atol=1e-9)


def test_nfft_level_matches_ndft_and_converges_to_direct():
    wl = workloads.tiny(N=400, d=3, seed=32, ell=[0.3])
    v = wl.vector().astype(np.float64)
    Kd, dKd = fastsum.direct_matern(wl.points, wl.windows, wl.ell, wl.sigma_f, v)
    errs = []
    for M in (16, 32, 64):
        Kn, dKn = fastsum.matvec_all(wl.points, wl.windows, wl.ell, wl.sigma_f, v, M, 4, kernel="matern")
        Kt, dKt = fastsum.matvec_all(wl.points, wl.windows, wl.ell, wl.sigma_f, v, M, 4, kernel="matern",
                                     level="ndft")
        assert np.linalg.norm(Kn - Kt) <= 1e-5 * np.linalg.norm(Kt)       # window error only
        errs.append(np.linalg.norm(Kt - Kd) / np.linalg.norm(Kd))
    assert errs[0] > errs[1] > errs[2]                                    # Fourier error shrinks with M
