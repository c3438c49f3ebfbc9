"""The pins have teeth: plant plausible mistakes in the oracle (CPU only) and check that
the corresponding pin would fail."""
import numpy as np

from oracle import fastsum, kernels, window


def rel(a, b):
    return np.linalg.norm(np.ravel(a - b)) / np.linalg.norm(np.ravel(b))


def _adjoint_err(x, v, M):
    return rel(fastsum.nfft_adjoint(x, v, M, 2 * M, 4), fastsum.adjoint_exact(x, v, M))


def test_wrong_deconvolution_is_caught(monkeypatch):
    rng = np.random.default_rng(0)
    x = rng.uniform(-0.2, 0.2, (100, 2))
    v = rng.standard_normal(100)
    assert _adjoint_err(x, v, 16) < 3e-6
    real = fastsum._phihat_grid
    monkeypatch.setattr(fastsum, "_phihat_grid", lambda M, n, m, s, d, win="kb": real(M, n, m, s, d, win) * (1 + 1e-3 * np.arange(M)[:, None]))
    assert _adjoint_err(x, v, 16) > 1e-4


def test_transposed_coordinates_are_caught():
    rng = np.random.default_rng(1)
    x = rng.uniform(-0.2, 0.2, (100, 2))
    v = rng.standard_normal(100)
    S = fastsum.adjoint_exact(x, v, 16)
    assert rel(fastsum.nfft_adjoint(x[:, ::-1].copy(), v, 16, 32, 4), S) > 1e-2


def test_conjugated_exponent_is_caught():
    rng = np.random.default_rng(2)
    x = rng.uniform(-0.2, 0.2, (100, 1))
    v = rng.standard_normal(100)
    S = fastsum.adjoint_exact(x, v, 16)
    assert rel(np.conj(fastsum.nfft_adjoint(x, v, 16, 32, 4)), S) > 1e-2


def test_dropped_half_in_derivative_kernel_is_caught(monkeypatch):
    """kappa_der with r^2/ell^2 instead of r^2/(2 ell^2) breaks the ell-derivative identity."""
    M, ell, h = 16, 0.5, 1e-5
    fd = (kernels.coefficients(ell + h, 3, M, 2, 1 / 16) - kernels.coefficients(ell - h, 3, M, 2, 1 / 16)) / (2 * h)
    good = kernels.coefficients(ell, 3, M, 2, 1 / 16, "der")
    assert np.abs(good - ell / 2 * fd).max() < 1e-9 * np.abs(good).max()
    real = kernels.kappa

    def bad(r, ell, kind="gauss"):
        return 2 * real(r, ell, kind) if kind == "der" else real(r, ell, kind)
    monkeypatch.setattr(kernels, "kappa", bad)
    worse = kernels.coefficients(ell, 3, M, 2, 1 / 16, "der")
    assert np.abs(worse - ell / 2 * fd).max() > 0.1 * np.abs(good).max()


def test_window_transform_mismatch_is_caught(monkeypatch):
    """Deconvolving by the transform of a different window (shape for sigma = 1.5) than the one the
    grid was spread with breaks the NFFT level."""
    rng = np.random.default_rng(3)
    x = rng.uniform(-0.2, 0.2, (100, 1))
    v = rng.standard_normal(100)
    assert _adjoint_err(x, v, 32) < 3e-6
    real = window.phihat_quadrature
    monkeypatch.setattr(window, "phihat_quadrature", lambda k, n, m, sigma=2.0, **kw: real(k, n, m, 1.5, **kw))
    fastsum._phihat_grid.cache_clear()          # the oracle keeps window transforms per setting
    try:
        assert _adjoint_err(x, v, 32) > 1e-3
    finally:
        fastsum._phihat_grid.cache_clear()


def test_unhalved_extension_coefficients_are_caught(monkeypatch):
    """Forgetting to split b_k between c_{+k} and c_{-k} doubles every non-constant term: the exact
    reproduction of a cosine polynomial fails."""
    M, a = 16, 0.3
    f = lambda x: 0.3 + 0.5 * np.cos(2 * np.pi * 3 * x)
    x = kernels.extension_nodes(a, M)
    good = kernels.cosine_extension(f(x), a, M)
    assert abs(good[M // 2 + 3] - 0.25) < 1e-9
    real = kernels.cosine_extension

    def bad(values, a, M):
        c = real(values, a, M)
        c[np.arange(M) != M // 2] *= 2
        return c
    monkeypatch.setattr(kernels, "cosine_extension", bad)
    worse = kernels.cosine_extension(f(x), a, M)
    assert abs(worse[M // 2 + 3] - 0.25) > 0.1


def test_dropped_term_of_the_derivative_sum_is_caught():
    """The derivative kernel's coefficients are a d-term sum (Sec. 3.4); dropping the last term breaks
    the agreement with kappa_der on the coordinate box."""
    M, ell, iv = 16, 0.5, [0.3, 0.3, 0.3]
    rng = np.random.default_rng(8)
    r = rng.uniform(-0.3, 0.3, (500, 3))
    want = kernels.kappa(np.linalg.norm(r, axis=1), ell, "der")
    good = kernels.coefficients_separable(ell, M, iv, "der")
    assert np.abs(kernels.trig_poly_eval(good, r) - want).max() < 1e-4
    f = [kernels.factor_coefficients(ell, a, M, "gauss") for a in iv]
    g = [kernels.factor_coefficients(ell, a, M, "der") for a in iv]
    o = np.multiply.outer
    two_terms = o(o(g[0], f[1]), f[2]) + o(o(f[0], g[1]), f[2])
    assert np.abs(kernels.trig_poly_eval(two_terms, r) - want).max() > 1e-2
