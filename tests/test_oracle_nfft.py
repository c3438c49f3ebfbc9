"""Pins for the oracle's fast summation levels (Sec. 3.1 eq. "approx fast sum"; Sec. 3.4
Hoelder bound eq. "NFFT approx error"; Sec. 3.4.4 error decomposition)."""
import numpy as np
import pytest

import workloads
from oracle import fastsum, kernels


def rel(a, b):
    return np.linalg.norm(np.ravel(a - b)) / np.linalg.norm(np.ravel(b))


@pytest.fixture(scope="module")
def pts3():
    wl = workloads.make("c0", N=600)
    return wl.points.astype(np.float64), wl.vector().astype(np.float64)


@pytest.mark.parametrize("win", ["kb", "es"])
@pytest.mark.parametrize("d", [1, 2, 3])
def test_adjoint_nfft_vs_exact(d, win):
    """Spread + FFT + deconvolution reproduces S_k = sum_j v_j exp(-2 pi i k.x_j) (the inner sums),
    with either window."""
    rng = np.random.default_rng(d)
    x = rng.uniform(-0.22, 0.22, size=(300, d))
    v = rng.standard_normal(300)
    M = 16 if d == 3 else 32
    S = fastsum.adjoint_exact(x, v, M)
    for m, tol in ((4, 3e-6), (6, 3e-10)):
        Sa = fastsum.nfft_adjoint(x, v, M, 2 * M, m, win=win)
        assert rel(Sa, S) < tol


@pytest.mark.parametrize("win", ["kb", "es"])
@pytest.mark.parametrize("d", [1, 2, 3])
def test_forward_nfft_vs_exact(d, win):
    """Deconvolution + zero-padded inverse FFT + interpolation reproduces sum_k d_k exp(2 pi i k.x),
    with either window."""
    rng = np.random.default_rng(10 + d)
    x = rng.uniform(-0.22, 0.22, size=(300, d))
    M = 16 if d == 3 else 32
    dh = rng.standard_normal((M,) * d) + 1j * rng.standard_normal((M,) * d)
    f = fastsum.forward_exact(x, dh).real
    for m, tol in ((4, 3e-6), (6, 3e-10)):
        assert rel(fastsum.nfft_forward(x, [dh], 2 * M, m, win=win)[0], f) < tol


def test_es_and_kb_fast_sums_agree(pts3):
    """The two windows approximate the same trigonometric sum: their fused products differ by no more
    than the sum of their window errors."""
    wl_pts, v = pts3
    c = kernels.coefficients(0.5, 3, 32, 2, 1 / 16)
    ref = fastsum.ndft_fastsum(wl_pts, v, [c])[0]
    kb = fastsum.nfft_fastsum(wl_pts, v, [c], 64, 4)[0]
    es = fastsum.nfft_fastsum(wl_pts, v, [c], 64, 4, win="es")[0]
    assert rel(es, ref) < 1e-6 and rel(kb, ref) < 1e-6
    assert rel(es, kb) <= rel(es, ref) + rel(kb, ref)


def test_window_error_decays_with_cutoff(pts3):
    x, v = pts3
    c = kernels.coefficients(0.5, 3, 16, 1, 1 / 16)
    ref = fastsum.ndft_fastsum(x, v, [c])[0]
    errs = [rel(fastsum.nfft_fastsum(x, v, [c], 32, m)[0], ref) for m in (2, 3, 4, 5)]
    assert all(b < a / 20 for a, b in zip(errs, errs[1:])), errs
    assert errs[2] < 1e-6


def test_nfft_operator_is_symmetric(pts3):
    """Real, even c_hat make the NFFT fast-sum operator symmetric: w^T K~ v = v^T K~ w to rounding."""
    x, v = pts3
    w = np.random.default_rng(5).standard_normal(len(v))
    for kind in ("gauss", "der"):
        c = kernels.coefficients(0.4, 3, 32, 2, 1 / 16, kind)
        Kv = fastsum.nfft_fastsum(x, v, [c], 64, 4)[0]
        Kw = fastsum.nfft_fastsum(x, w, [c], 64, 4)[0]
        assert abs(w @ Kv - v @ Kw) <= 1e-12 * np.abs(w) @ np.abs(Kv)


def test_three_point_normalisation():
    """With three points the NFFT fast sum equals the trigonometric sum built directly from its
    definition term by term (fixes the n^d and phi_hat normalisation)."""
    x = np.array([[0.1, -0.05, 0.02], [-0.2, 0.1, 0.0], [0.0, 0.0, 0.15]])
    v = np.array([1.0, -2.0, 0.5])
    M = 16
    c = kernels.coefficients(0.3, 3, M, 1, 1 / 16)
    k = np.arange(-M // 2, M // 2)
    K = np.stack(np.meshgrid(k, k, k, indexing="ij"), -1).reshape(-1, 3)
    cf = c.reshape(-1)
    exact = np.array([sum(v[j] * np.sum(cf * np.cos(2 * np.pi * K @ (x[i] - x[j]))) for j in range(3))
                      for i in range(3)])
    np.testing.assert_allclose(fastsum.nfft_fastsum(x, v, [c], 2 * M, 6)[0], exact, rtol=1e-9, atol=1e-9)


def test_hoelder_bound(pts3):
    """|h(x_i) - h~(x_i)| <= ||v||_1 ||K_R - K_F||_inf (eq. "NFFT approx error"), the sup taken over
    all differences x_i - x_j that can occur (here estimated on a dense sample of the ball of
    radius 1/2 - eps_B plus the actual differences)."""
    x, v = pts3
    ell, M, p = 0.5, 32, 2
    c = kernels.coefficients(ell, 3, M, p, 1 / 16)
    h_direct, _ = fastsum.direct(x.astype(np.float32), [(0, 1, 2)], [ell], 1.0, v)
    h_trig = fastsum.ndft_fastsum(x, v, [c])[0]
    rng = np.random.default_rng(9)
    r = rng.standard_normal((20000, 3))
    r *= (0.4375 * rng.uniform(0, 1, (20000, 1)) ** (1 / 3)) / np.linalg.norm(r, axis=1, keepdims=True)
    r = np.vstack([r, (x[:40, None, :] - x[None, :, :]).reshape(-1, 3)])
    sup = np.abs(kernels.trig_poly_eval(c, r) - kernels.kappa(np.linalg.norm(r, axis=1), ell)).max()
    assert np.all(np.abs(h_direct - h_trig) <= np.abs(v).sum() * sup * 1.0001 + 1e-12)


def test_end_to_end_c0_levels():
    """Config c0 (N=2000): CPU NFFT -> NDFT within the window error; NDFT -> direct at the Fourier
    error of the method at M=32 (measured 1.1e-3 for K v and 5.3e-3 for the derivative product;
    the per-output Hoelder bound above is the guarantee, these limits guard against regressions)."""
    wl = workloads.make("c0")
    v = wl.vector().astype(np.float64)
    Kd, dKd = fastsum.direct(wl.points, wl.windows, wl.ell, wl.sigma_f, v)
    Kn, dKn = fastsum.matvec_all(wl.points, wl.windows, wl.ell, wl.sigma_f, v, 32, 4)
    Kt, dKt = fastsum.matvec_all(wl.points, wl.windows, wl.ell, wl.sigma_f, v, 32, 4, level="ndft")
    assert rel(Kn, Kt) < 1e-6 and rel(dKn, dKt) < 1e-6
    assert rel(Kt, Kd) < 1.5e-3 and rel(dKt, dKd) < 7e-3


def test_large_ell_and_fine_grid_converge_to_direct():
    """With a wide kernel (ell = 3) the radially regularised periodisation is nearly smooth and the fast
    sum meets the direct sum closely; M = 64 is more accurate than M = 32."""
    wl = workloads.make("c0", N=500)
    v = wl.vector().astype(np.float64)
    Kd, _ = fastsum.direct(wl.points, wl.windows, [3.0], 1.0, v)
    K32, _ = fastsum.matvec_all(wl.points, wl.windows, [3.0], 1.0, v, 32, 4, reg="radial")
    K64, _ = fastsum.matvec_all(wl.points, wl.windows, [3.0], 1.0, v, 64, 4, reg="radial")
    assert rel(K64, Kd) < rel(K32, Kd) < 1e-4


def test_sigma_f_and_derivative_scalings():
    """matvec_all applies sigma_f^2 to K v and sigma_f^2 (2/ell_s) to K_s^der v (Sec. 3.3)."""
    wl = workloads.tiny(N=50, d=6, windows=[(0, 1, 2), (3, 4, 5)], ell=[0.3, 0.6])
    v = wl.vector().astype(np.float64)
    K1, D1 = fastsum.matvec_all(wl.points, wl.windows, wl.ell, 1.0, v, 16, 4)
    K2, D2 = fastsum.matvec_all(wl.points, wl.windows, wl.ell, 2.5, v, 16, 4)
    np.testing.assert_allclose(K2, 6.25 * K1, rtol=1e-13)
    np.testing.assert_allclose(D2, 6.25 * D1, rtol=1e-13)
    X = wl.points.astype(np.float64)
    for s, w in enumerate(wl.windows):
        xs = np.ascontiguousarray(X[:, list(w)])
        _, cd, q = fastsum.coefficients_for(xs, wl.ell[s], 16)
        raw = fastsum.nfft_fastsum(xs, v, [cd], 32, 4)[0] + q * kernels.quadratic_part(xs, v)
        np.testing.assert_allclose(D1[s], 2.0 / wl.ell[s] * raw, rtol=1e-13)


def test_row_subset_matches_full():
    """Evaluating the fast sum at a subset of targets gives exactly those rows of the full result."""
    wl = workloads.make("c1", N=3000)
    v = wl.vector().astype(np.float64)
    K, D = fastsum.matvec_all(wl.points, wl.windows, wl.ell, wl.sigma_f, v, wl.bandwidth, wl.cutoff)
    rows = np.array([5, 0, 2999, 1234])
    Kr, Dr = fastsum.matvec_all(wl.points, wl.windows, wl.ell, wl.sigma_f, v, wl.bandwidth, wl.cutoff, rows=rows)
    np.testing.assert_allclose(Kr, K[rows], rtol=1e-14, atol=1e-14)
    np.testing.assert_allclose(Dr, D[:, rows], rtol=1e-14, atol=1e-14)
