"""Pins for the oracle's window transform, kernels, regularisation and discrete
Fourier coefficients (Sec. 3.1, Lemma "aliasing error", Sec. 3.4 tensor forms)."""
import mpmath as mp
import numpy as np
import pytest

from oracle import bounds, kernels, window


# ---------------------------------------------------------------- window ----

@pytest.mark.parametrize("n,m", [(32, 4), (64, 4), (64, 3), (128, 6)])
def test_phihat_quadrature_vs_closed_form(n, m):
    """The quadrature of the truncated window against the published closed form I_0(...)/n.
    The closed form is the transform of the untruncated window; the part cut off beyond |n x| = m
    is smaller than phi_hat(0) by about exp(-b m), which sets the tolerance."""
    M = n // 2
    k = np.arange(-M // 2, M // 2)
    q = window.phihat_quadrature(k, n, m)
    c = window.phihat_closed_form(k, n, m)
    np.testing.assert_allclose(q, c, rtol=max(2 * np.exp(-window.shape(2.0) * m), 1e-11))


def test_phihat_quadrature_high_precision():
    """Against a 30-digit mpmath quadrature of the same definition."""
    mp.mp.dps = 30
    n, m = 64, 4
    b = mp.pi * mp.mpf(3) / 2
    for k in (0, 7, 16):
        f = lambda x: (mp.sinh(b * mp.sqrt(m * m - (n * x) ** 2)) / (mp.pi * mp.sqrt(m * m - (n * x) ** 2))
                       * mp.cos(2 * mp.pi * k * x))
        ref = float(mp.quad(f, [-mp.mpf(m) / n, 0, mp.mpf(m) / n]))
        assert window.phihat_quadrature([k], n, m)[0] == pytest.approx(ref, rel=1e-12)


def test_window_partition_of_unity():
    """Poisson summation: sum_l phi(x - l/n) = n sum_r phi_hat(r n) e^{2 pi i r n x} ~= n phi_hat(0)."""
    n, m = 64, 4
    x = np.random.default_rng(0).uniform(-0.5, 0.5, 50)
    l = np.arange(-n // 2 - 8, n // 2 + 8)
    s = window.phi(x[:, None] - l[None, :] / n, n, m).sum(axis=1)
    np.testing.assert_allclose(s, n * window.phihat_quadrature([0], n, m)[0], rtol=1e-6)


def test_window_shape():
    n, m = 64, 4
    x = np.linspace(-0.1, 0.1, 1001)
    p = window.phi(x, n, m)
    np.testing.assert_allclose(p, p[::-1], rtol=1e-12)
    assert np.all(p[np.abs(x) > m / n] == 0) and np.all(p[np.abs(x) <= m / n] > 0)
    assert p.argmax() == 500


def test_es_phihat_quadrature_high_precision():
    """Exponential-of-semicircle window: the transform against a 30-digit mpmath (tanh-sinh) quadrature
    of its definition exp(beta (sqrt(1 - (n x/m)^2) - 1)), beta = 2.30 * 2m at sigma = 2."""
    mp.mp.dps = 30
    n, m = 64, 4
    beta = mp.mpf("2.30") * 2 * m
    assert window.es_beta(m) == pytest.approx(float(beta), rel=1e-15)
    for k in (0, 7, 16, 31):
        f = lambda x: mp.exp(beta * (mp.sqrt(1 - (n * x / m) ** 2) - 1)) * mp.cos(2 * mp.pi * k * x)
        ref = float(mp.quad(f, [-mp.mpf(m) / n, 0, mp.mpf(m) / n]))
        assert window.phihat_quadrature([k], n, m, window="es")[0] == pytest.approx(ref, rel=1e-10)


def test_es_window_shape_and_partition_of_unity():
    """ES window: even, peak 1 at the centre, exp(-beta) at the edge of its support, zero outside; and
    its shifts sum to n phi_hat(0) up to the aliasing of phi_hat at multiples of n (Poisson summation)."""
    n, m = 64, 4
    x = np.linspace(-0.1, 0.1, 1001)
    p = window.phi(x, n, m, window="es")
    np.testing.assert_allclose(p, p[::-1], rtol=1e-12)
    assert p[500] == 1.0 and np.all(p[np.abs(x) > m / n] == 0)
    assert window.phi([m / n], n, m, window="es")[0] == pytest.approx(np.exp(-window.es_beta(m)), rel=1e-12)
    xs = np.random.default_rng(0).uniform(-0.5, 0.5, 50)
    l = np.arange(-n // 2 - 8, n // 2 + 8)
    s = window.phi(xs[:, None] - l[None, :] / n, n, m, window="es").sum(axis=1)
    np.testing.assert_allclose(s, n * window.phihat_quadrature([0], n, m, window="es")[0], rtol=1e-6)


# ---------------------------------------------------------------- kernels ---

def test_kernel_closed_forms():
    """kappa_der = (ell/2) d kappa_gauss / d ell (Sec. 3.3: K_der = ell/2 K^ell), checked by an
    high-precision numerical derivative; and kappa_der = 1/2 (kappa + ell^2 kappa'') (Sec. 3.1)."""
    r = np.linspace(0, 0.6, 31)
    for ell in (0.1, 0.5, 2.0):
        dl = np.array([float(mp.diff(lambda L: mp.exp(-float(t) ** 2 / (2 * L * L)), ell)) for t in r])
        np.testing.assert_allclose(kernels.kappa(r, ell, "der"), ell / 2 * dl, rtol=1e-10, atol=1e-14)
        d2 = np.array([float(mp.diff(lambda t: mp.exp(-t * t / (2 * ell * ell)), float(t), 2)) for t in r])
        np.testing.assert_allclose(kernels.kappa(r, ell, "der"), 0.5 * (kernels.kappa(r, ell) + ell ** 2 * d2),
                                   rtol=1e-10, atol=1e-14)


@pytest.mark.parametrize("kind", ["gauss", "der"])
def test_radial_derivatives_vs_mpmath(kind):
    for ell in (0.12, 0.5, 1.3):
        a = 0.4375
        got = kernels.radial_derivatives(a, ell, 6, kind)
        f = ((lambda t: mp.exp(-t * t / (2 * ell * ell))) if kind == "gauss"
             else (lambda t: t * t / (2 * ell * ell) * mp.exp(-t * t / (2 * ell * ell))))
        ref = [float(mp.diff(f, a, j)) for j in range(6)]
        np.testing.assert_allclose(got, ref, rtol=1e-10, atol=1e-12)


@pytest.mark.parametrize("p", [1, 2, 4, 8])
@pytest.mark.parametrize("kind", ["gauss", "der"])
def test_regularisation_conditions(p, kind):
    """K_R = kappa on r <= a; the transition polynomial matches kappa's first p derivatives at a,
    reaches kappa(1/2) at 1/2 with p-1 vanishing derivatives; constant beyond 1/2."""
    eps_B = 1 / 16
    a = 0.5 - eps_B
    for ell in (0.2, 0.5, 1.0):
        r = np.linspace(0, a, 200)
        np.testing.assert_array_equal(kernels.regularised(r, ell, p, eps_B, kind), kernels.kappa(r, ell, kind))
        t = kernels.transition_polynomial(ell, p, eps_B, kind)
        poly = np.polynomial.Polynomial(t)
        f = ((lambda s: mp.exp(-s * s / (2 * ell * ell))) if kind == "gauss"
             else (lambda s: s * s / (2 * ell * ell) * mp.exp(-s * s / (2 * ell * ell))))
        for j in range(p):
            assert poly.deriv(j)(0.0) == pytest.approx(float(mp.diff(f, a, j)), rel=1e-9, abs=1e-10)
            at_half = poly.deriv(j)(eps_B)
            assert at_half == pytest.approx(float(f(0.5)) if j == 0 else 0.0, abs=1e-9 * max(1, abs(t).max()))
        beyond = kernels.regularised(np.array([0.51, 0.7, 0.86]), ell, p, eps_B, kind)
        np.testing.assert_array_equal(beyond, float(kernels.kappa(0.5, ell, kind)))


# ---------------------------------------------------------- coefficients ----

@pytest.mark.parametrize("M", [16, 32])
@pytest.mark.parametrize("ell", [0.1, 0.3, 0.8])
def test_1d_coefficients_aliasing_formula(M, ell):
    """Lemma "aliasing error": c_hat_k = sum_r c_{k + M r} with the analytic c_k of the plain
    periodic continuation (Sec. 3.1, complex-erf form)."""
    chat = kernels.coefficients(ell, 1, M, 0, 1 / 16)
    k = np.arange(-M // 2, M // 2)
    R = 40000
    r = np.arange(-R, R + 1)
    alias = np.array([bounds.analytic_coeff_gauss_1d(kk + M * r, ell).sum() for kk in k])
    np.testing.assert_allclose(chat, alias, rtol=0, atol=2e-7)


def test_1d_analytic_coefficients_by_quadrature():
    for ell in (0.1, 0.4, 1.5):
        for k in (0, 1, 5, 17):
            ref = float(mp.quad(lambda x: mp.exp(-x * x / (2 * ell * ell)) * mp.cos(2 * mp.pi * k * x), [-0.5, 0.5]))
            assert bounds.analytic_coeff_gauss_1d(k, ell) == pytest.approx(ref, rel=1e-10, abs=1e-15)


@pytest.mark.parametrize("d", [2, 3])
def test_tensor_product_structure(d):
    """Without regularisation the d-variate Gaussian separates, so c_hat_k = prod_t c_hat_{k_t}
    (Sec. 3.4.1); the derivative kernel gives the three-term sum of Sec. 3.4.2."""
    M, ell = 16, 0.35
    cg = kernels.coefficients(ell, d, M, 0, 1 / 16, "gauss")
    cd = kernels.coefficients(ell, d, M, 0, 1 / 16, "der")
    f1 = kernels.coefficients(ell, 1, M, 0, 1 / 16, "gauss")
    g1 = kernels.coefficients(ell, 1, M, 0, 1 / 16, "der")
    if d == 2:
        np.testing.assert_allclose(cg, np.multiply.outer(f1, f1), atol=1e-15)
        np.testing.assert_allclose(cd, np.multiply.outer(g1, f1) + np.multiply.outer(f1, g1), atol=1e-15)
    else:
        o = lambda a, b, c: np.multiply.outer(np.multiply.outer(a, b), c)
        np.testing.assert_allclose(cg, o(f1, f1, f1), atol=1e-15)
        np.testing.assert_allclose(cd, o(g1, f1, f1) + o(f1, g1, f1) + o(f1, f1, g1), atol=1e-15)


def test_coefficients_real_even():
    c = kernels.coefficients(0.4, 3, 16, 2, 1 / 16, "der")
    inner = c[1:, 1:, 1:]
    np.testing.assert_allclose(inner, inner[::-1, ::-1, ::-1], atol=1e-15)
    np.testing.assert_allclose(inner, inner.transpose(1, 0, 2), atol=1e-15)


@pytest.mark.parametrize("p", [0, 2, 4])
def test_der_coefficients_are_ell_derivative(p):
    """Because the regularisation is linear in the kernel's data at a and at 1/2, regularising
    kappa_der gives (ell/2) d/d ell of the regularised kappa, coefficient by coefficient."""
    M, d, eps_B = 16, 3, 1 / 16
    for ell in (0.3, 0.9):
        h = 1e-5 * ell
        fd = (kernels.coefficients(ell + h, d, M, p, eps_B) - kernels.coefficients(ell - h, d, M, p, eps_B)) / (2 * h)
        cd = kernels.coefficients(ell, d, M, p, eps_B, "der")
        np.testing.assert_allclose(cd, ell / 2 * fd, atol=1e-9 * np.abs(cd).max())


def test_trig_poly_interpolates_samples():
    """K_F(j/M) equals the sample K_R(||j/M||) on the grid (the DFT is invertible)."""
    M, ell, p = 16, 0.4, 2
    c = kernels.coefficients(ell, 3, M, p, 1 / 16)
    rng = np.random.default_rng(3)
    j = rng.integers(-M // 2, M // 2, size=(40, 3)) / M
    np.testing.assert_allclose(kernels.trig_poly_eval(c, j),
                               kernels.regularised(np.linalg.norm(j, axis=1), ell, p, 1 / 16), atol=1e-13)
